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

// the same slot with one padding element after every 2^pshift slots (pshift
// >= 31: no padding).  The real-to-complex row phase reads the transform at
// bit-reversed positions: consecutive frequencies then sit 2^(log n - 5)
// slots apart, and this padding spreads them over the banks.
__device__ __forceinline__ int fslotp(int s, int e, int cnt, int pshift)
{
    const int p = fslot(s, e, cnt);
    return p + (p >> pshift);
}

// stages s0 .. s0+L-1 (DIF: the highest first)
template <int L, bool DIF>
__device__ __forceinline__ void fft_pass(float2 *a, int n, int cnt, int lcnt, const float2 *__restrict__ tw,
                                         bool inv, int s0, int pshift)
{
    constexpr int R = 1 << L;
    const int h = 1 << (s0 - 1), total = cnt * (n >> L);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int sq = t & (cnt - 1), it = t >> lcnt;
        const int k = it & (h - 1), base = ((it >> (s0 - 1)) << (s0 - 1 + L)) + k;
        // the pass's twiddles first (stage s0 + ll uses w^(k + mm h), mm < 2^ll,
        // at table stride n >> (s0 + ll)), so that their loads overlap
        float2 w[R - 1];
#pragma unroll
        for (int ll = 0; ll < L; ++ll)
#pragma unroll
            for (int mm = 0; mm < (1 << ll); ++mm) {
                float2 x = __ldg(tw + (k + mm * h) * (n >> (s0 + ll)));
                if (inv) x.y = -x.y;
                w[(1 << ll) - 1 + mm] = x;
            }
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = a[fslotp(sq, base + m * h, cnt, pshift)];
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int ll = DIF ? (L - 1 - l) : l;   // stage s0 + ll, distance dl (in units of h)
            const int dl = 1 << ll;
#pragma unroll
            for (int m = 0; m < R; ++m) {
                if (m & dl) continue;
                const float2 w_ = w[dl - 1 + (m & (dl - 1))];
                const float2 u = v[m], x = v[m + dl];
                if (DIF) {
                    v[m] = make_float2(u.x + x.x, u.y + x.y);
                    v[m + dl] = cmul(make_float2(u.x - x.x, u.y - x.y), w_);
                } else {
                    const float2 xw = cmul(x, w_);
                    v[m] = make_float2(u.x + xw.x, u.y + xw.y);
                    v[m + dl] = make_float2(u.x - xw.x, u.y - xw.y);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < R; ++m) a[fslotp(sq, base + m * h, cnt, pshift)] = v[m];
    }
    __syncthreads();
}

// Pass plan of the real-to-complex phases: np = ceil(logn / 3) passes; in
// decimation-in-time order pass 0 takes stages 1 .. L0 (L0 = logn - 3 (np-1))
// and pass i > 0 stages L0 + 3(i-1) + 1 .. L0 + 3i; decimation in frequency
// runs the same passes from the last to the first.  So the last inverse pass
// and the first forward pass cover the same stages and give every thread the
// same elements: an element-wise step between an inverse and a forward
// transform needs no trip through shared memory.
__host__ __device__ __forceinline__ int fft_npass(int logn) { return (logn + 2) / 3; }
__host__ __device__ __forceinline__ int fft_pass_len(int logn, int i) { return i == 0 ? logn - 3 * (fft_npass(logn) - 1) : 3; }
__host__ __device__ __forceinline__ int fft_pass_s0(int logn, int i) { return i == 0 ? 1 : fft_pass_len(logn, 0) + 3 * (i - 1) + 1; }

// One pass of radix-2 stages s0 .. s0+L-1 (butterflies at distance
// h = 2^(s0-1)) over cnt transforms of length n.  Group t of the pass holds
// elements e_m = base + m h (m < 2^L) of transform sq = t mod cnt;
// ld(sq, e, m) supplies an element and st(sq, e, m, v) takes it.  MODE 0: the
// stages decimation in frequency (forward); 1: decimation in time with
// conjugate twiddles (unscaled inverse); 2: the inverse stages, then
// mid(sq, base, h, v) on the 2^L values in registers, then the forward
// stages; 3: forward, mid, inverse.  The arithmetic of each stage is that of
// fft_pass.  No barrier.
template <int L, int MODE, typename Ld, typename Mid, typename St>
__device__ __forceinline__ void fft_pass_g(int n, int cnt, int lcnt, const float2 *__restrict__ tw, int s0, Ld ld,
                                           Mid mid, St st)
{
    constexpr int R = 1 << L;
    const int h = 1 << (s0 - 1), total = cnt * (n >> L);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int sq = t & (cnt - 1), it = t >> lcnt;
        const int k = it & (h - 1), base = ((it >> (s0 - 1)) << (s0 - 1 + L)) + k;
        // the pass's twiddles: stage s0 + ll uses w^(k + mm h) = w^k exp(-i pi mm / 2^ll)
        // (mm < 2^ll), so one table value per stage; the factors -i are
        // exact, exp(-i pi / 4) and exp(-3 i pi / 4) cost one rounding
        float2 w[R - 1];
#pragma unroll
        for (int ll = 0; ll < L; ++ll) {
            const float2 b0 = __ldg(tw + k * (n >> (s0 + ll)));
            w[(1 << ll) - 1] = b0;
            if (ll >= 1) w[(1 << ll) - 1 + (1 << (ll - 1))] = make_float2(b0.y, -b0.x);   // times -i
            if (ll == 2) {
                const float c = 0.70710678118654752f;   // 1/sqrt(2)
                w[4] = make_float2(c * (b0.x + b0.y), c * (b0.y - b0.x));   // times (1 - i)/sqrt(2)
                w[6] = make_float2(c * (b0.y - b0.x), -c * (b0.x + b0.y));  // times (-1 - i)/sqrt(2)
            }
        }
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = ld(sq, base + m * h, m);
        auto dit = [&]() {
#pragma unroll
            for (int ll = 0; ll < L; ++ll) {
                const int dl = 1 << ll;
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    if (m & dl) continue;
                    float2 w_ = w[dl - 1 + (m & (dl - 1))];
                    w_.y = -w_.y;
                    const float2 u = v[m], xw = cmul(v[m + dl], w_);
                    v[m] = make_float2(u.x + xw.x, u.y + xw.y);
                    v[m + dl] = make_float2(u.x - xw.x, u.y - xw.y);
                }
            }
        };
        auto dif = [&]() {
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const int ll = L - 1 - l, dl = 1 << ll;
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    if (m & dl) continue;
                    const float2 w_ = w[dl - 1 + (m & (dl - 1))];
                    const float2 u = v[m], x = v[m + dl];
                    v[m] = make_float2(u.x + x.x, u.y + x.y);
                    v[m + dl] = cmul(make_float2(u.x - x.x, u.y - x.y), w_);
                }
            }
        };
        if constexpr (MODE == 0) dif();
        if constexpr (MODE == 1) dit();
        if constexpr (MODE == 2) { dit(); mid(sq, base, h, v); dif(); }
        if constexpr (MODE == 3) { dif(); mid(sq, base, h, v); dit(); }
#pragma unroll
        for (int m = 0; m < R; ++m) st(sq, base + m * h, m, v[m]);
    }
}

// fft_pass_g with the pass length chosen at run time (1, 2 or 3 stages)
template <int MODE, typename Ld, typename Mid, typename St>
__device__ __forceinline__ void fft_pass_n(int L, int n, int cnt, int lcnt, const float2 *__restrict__ tw, int s0, Ld ld,
                                           Mid mid, St st)
{
    if (L == 3) fft_pass_g<3, MODE>(n, cnt, lcnt, tw, s0, ld, mid, st);
    else if (L == 2) fft_pass_g<2, MODE>(n, cnt, lcnt, tw, s0, ld, mid, st);
    else fft_pass_g<1, MODE>(n, cnt, lcnt, tw, s0, ld, mid, st);
}

// all logn stages: DIF (forward use: natural -> bit-reversed) or DIT
// (bit-reversed -> natural); inv conjugates the twiddles
template <bool DIF>
__device__ __forceinline__ void fft_stages(float2 *a, int n, int logn, int cnt, const float2 *__restrict__ tw, bool inv,
                                           int pshift = 31)
{
    const int lcnt = __ffs(cnt) - 1;
    for (int done = 0; done < logn;) {
        const int L = logn - done < 3 ? logn - done : 3;
        const int s0 = DIF ? logn - done - L + 1 : done + 1;
        if (L == 3) fft_pass<3, DIF>(a, n, cnt, lcnt, tw, inv, s0, pshift);
        else if (L == 2) fft_pass<2, DIF>(a, n, cnt, lcnt, tw, inv, s0, pshift);
        else fft_pass<1, DIF>(a, n, cnt, lcnt, tw, inv, s0, pshift);
        done += L;
    }
}

} // namespace adp
