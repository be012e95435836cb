// Radix-2 FFTs in shared memory for the FFT operator path of the engine.
//
// With periodic boundaries the operator of Eq. 2.4 is a circular convolution,
// B x = k * x with k(u, v) = b[u + r, v + r] (u, v taken modulo H and W), so
// by the convolution theorem F(B x) = F(k) . F(x) and F(B^T z) = conj(F(k)) . F(z)
// for real k.  The engine evaluates both with 2-D transforms of power-of-two
// sizes: a length-W transform per image row, a length-H transform per column.
//
// Forward transforms use decimation in frequency (Gentleman-Sande: natural
// order in, bit-reversed order out) and inverse transforms decimation in time
// (Cooley-Tukey: bit-reversed order in, natural order out).  The spectrum of
// the kernel is stored in the same bit-reversed order, so the pointwise
// product needs no permutation and none is ever made.
//
// `cnt` transforms of length n = 2^logn run together (cnt a power of two);
// element e of transform s lives at a[e * cnt + (s ^ (e & (cnt - 1)))], so a
// warp's lanes (consecutive s) touch consecutive words, and a row of the
// global image (consecutive e, fixed s) spreads over the banks.  Stage s
// (butterflies at distance h = 2^(s-1), group size 2h) multiplies by
// w^k = exp(-+2 pi i k / 2h), read from the table tw[j] = exp(-2 pi i j / n),
// j < n/2, at j = k n / 2h; the inverse conjugates w and leaves the 1/n
// scaling to the caller.  Up to three consecutive stages run per pass over
// shared memory, each thread holding the 2^L values they combine in
// registers; the arithmetic (and its rounding) is that of plain radix-2.
// Every thread of the CTA takes part; each pass ends with __syncthreads().
#pragma once

namespace adp {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// shared-memory slot of element e of transform s (cnt transforms)
__device__ __forceinline__ int fslot(int s, int e, int cnt) { return e * cnt + (s ^ (e & (cnt - 1))); }

// stages s0 .. s0+L-1 (DIF: the highest first)
template <int L, bool DIF>
__device__ __forceinline__ void fft_pass(float2 *a, int n, int cnt, int lcnt, const float2 *__restrict__ tw,
                                         bool inv, int s0)
{
    constexpr int R = 1 << L;
    const int h = 1 << (s0 - 1), total = cnt * (n >> L);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int sq = t & (cnt - 1), it = t >> lcnt;
        const int k = it & (h - 1), base = ((it >> (s0 - 1)) << (s0 - 1 + L)) + k;
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = a[fslot(sq, base + m * h, cnt)];
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int ll = DIF ? (L - 1 - l) : l;   // stage s0 + ll, distance dl (in units of h)
            const int dl = 1 << ll, tws = n >> (s0 + ll);
#pragma unroll
            for (int m = 0; m < R; ++m) {
                if (m & dl) continue;
                float2 w = __ldg(tw + (k + (m & (dl - 1)) * h) * tws);
                if (inv) w.y = -w.y;
                const float2 u = v[m], x = v[m + dl];
                if (DIF) {
                    v[m] = make_float2(u.x + x.x, u.y + x.y);
                    v[m + dl] = cmul(make_float2(u.x - x.x, u.y - x.y), w);
                } else {
                    const float2 xw = cmul(x, w);
                    v[m] = make_float2(u.x + xw.x, u.y + xw.y);
                    v[m + dl] = make_float2(u.x - xw.x, u.y - xw.y);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < R; ++m) a[fslot(sq, base + m * h, cnt)] = v[m];
    }
    __syncthreads();
}

// all logn stages: DIF (forward use: natural -> bit-reversed) or DIT
// (bit-reversed -> natural); inv conjugates the twiddles
template <bool DIF>
__device__ __forceinline__ void fft_stages(float2 *a, int n, int logn, int cnt, const float2 *__restrict__ tw, bool inv)
{
    const int lcnt = __ffs(cnt) - 1;
    for (int done = 0; done < logn;) {
        const int L = logn - done < 3 ? logn - done : 3;
        const int s0 = DIF ? logn - done - L + 1 : done + 1;
        if (L == 3) fft_pass<3, DIF>(a, n, cnt, lcnt, tw, inv, s0);
        else if (L == 2) fft_pass<2, DIF>(a, n, cnt, lcnt, tw, inv, s0);
        else fft_pass<1, DIF>(a, n, cnt, lcnt, tw, inv, s0);
        done += L;
    }
}

} // namespace adp
