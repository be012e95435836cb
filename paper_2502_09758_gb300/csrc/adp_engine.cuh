// The persistent engine of libadp: every phase of the hot path as a device
// member function and the cooperative kernel that runs one program of phases.
// Included by the per-precision translation units adp_f32.cu and adp_f64.cu.
//
// Data: the images of a call live in one padded workspace (see Ctx).  Periodic
// ghost rows and columns around each image are written together with the
// pixels they copy, so every tile a strip needs is a rectangular box that one
// TMA instruction (cp.async.bulk.tensor) stages into shared memory.  The
// caller's dense buffers are imported at the start of a call and exported at
// its end.
//
// Work decomposition: a strip is 32 columns x MR rows of one channel.  Strips
// are dealt to warps warp-major (strip s goes to warp s mod (grid * warps) in
// the order warp*grid + cta, so consecutive strips land on different SMs).  The
// correlation input of a strip is staged in stages of NX = PC + MR - 1 tile
// rows (the rows that PC kernel rows need), double-buffered per warp: lane 0
// issues stage k+1 on the warp's other mbarrier while the warp computes stage k.
//
// Convolution geometry (Eq. 2.4): (B x)[c,i,j] = sum_{p,q} b[c,p,q] x[c,i-p+r,j-q+r].
// With the tile origin at (row0-r, col0-r), B x is the correlation of the tile
// with the flipped kernel and B^T z the correlation with b as stored; both
// orientations are kept (rows zero-padded to Kp), in shared memory when they
// fit beside the warps' stages, else in a global slot read through L1.  Stage boxes start at column col0 - r4
// (r4 = r rounded up to 4, for 16-byte aligned boxes), so the correlation reads
// a stage from column offset r4 - r.
//
// Failure handling: a grid barrier that gives up returns false in every
// thread of its CTA (alive), and the programs unwind.  An mbarrier wait that
// gives up raises ST_TIMEOUT and stops that warp's TMA work for the rest of the
// launch (tmafail); the next grid barrier then fails everywhere.  Before the
// kernel returns, such a warp waits (bounded) for its copies in flight.
#pragma once

#include "adp_device.cuh"
#include "adp_fft.cuh"

#include <type_traits>

namespace adp {

// CTA-wide scratch of the engine in static shared memory (namespace scope, so
// that its addresses are constants rather than values held in registers).
// The reduction scalar S is 8 bytes (a float-float pair or a double).
__shared__ __align__(16) double g_red[MAXNW_FFT];
__shared__ __align__(16) double g_bcast[2];
__shared__ double g_redd[MAXNW_FFT];
__shared__ __align__(16) double g_tau[MAXC];
__shared__ __align__(16) double g_gbuf[GT_MAX];
__shared__ int g_sflag;
// each warp's two mbarriers (outside the warp regions, which the FFT phases
// reuse as one CTA-wide scratch area between passes)
__shared__ __align__(8) uint64_t g_mbar[MAXNW_FFT][2];
// the FFT phases' bulk copies: column stages 0 and 1, the row buffer
__shared__ __align__(8) uint64_t g_fmbar[3];

// Report of a MAID step, accumulated by thread 0 of each CTA (shared memory,
// so that it occupies no registers while the solves run).
struct MaidRep {
    int ll_iters, cg_iters, ll_capped, cg_capped, trials;
    long long fused;             // FISTA + CG iterations over the run
    double loss, gxn, znorm, psi;
};
__shared__ MaidRep g_rep;
// channel sums and means of the FFT kernel-gradient correlation (MAXC channels)
__shared__ double g_csum[4 * MAXC];
__shared__ double g_mx[MAXC], g_mv[MAXC];
__shared__ double g_xoff[MAXC];

// FFTP: compile the FFT operator path in (a separate instantiation, so that
// the direct program's register allocation does not carry it).
template <typename T, bool FFTP = false>
struct Eng {
    using Sc = Scal<T>;
    using S = typename Sc::S;      // reduction / control scalar (float-float or double)
    static constexpr int MR = Cfg<T>::MR;
    static constexpr int PC = Cfg<T>::PC;
    static constexpr int NX = PC + MR - 1;
    static constexpr int EWB = 4;  // element-wise phases: loads issued per batch per thread
    static constexpr bool kFFT = FFTP && std::is_same<T, float>::value;   // FFT path: FP32 only
    const Ctx<T> &cx;
    const Ctx<T> *mc;              // where the tensor maps live (parameter or global space)
    const T *wF, *wT;              // kernel orientations in use (shared memory or a global slot)
    T *wsm;                        // shared-memory home of both orientations (when cx.wsm)
    T *sb0;                        // this warp's region: stage buffers, halo-1 tiles, interior tile, mbarriers
    unsigned mph;                  // bit i: parity of mbar[i]'s next completion
    int wslot;                     // global weight slot written last
    int lane, warp;
    int nblk, bid;                 // CTAs sharing this program (grid or group) and this CTA's rank
    unsigned epoch;                // barriers passed so far (same in every thread)
    bool alive;                    // false once a grid barrier failed (uniform in the CTA)
    bool tmafail;                  // this warp gave up waiting for a TMA copy
    bool gedge;                    // the current strip has pixels whose copies live in the ghosts
    unsigned fph, fpend;           // g_fmbar: parity of each barrier's next completion; copies issued, not waited
    bool ffail;                    // a wait on g_fmbar gave up (uniform in the CTA)

    // the warp's region, derived from sb0 (Layout: two stages, two halo-1
    // tiles, an interior tile, the mbarriers)
    static constexpr int TILE1 = round_up((MR + 2) * 40, 32);
    static constexpr int TILEI = round_up(MR * 32, 32);
    // (the FFT instantiation has no direct correlation: no stages)
    __device__ int stage_elems() const { return kFFT ? 0 : round_up(NX * cx.BW, 32); }
    __device__ T *sb1() const { return sb0 + stage_elems(); }
    __device__ T *t1() const { return sb0 + 2 * stage_elems(); }
    __device__ T *t2() const { return t1() + TILE1; }
    __device__ T *tF() const { return t2() + TILE1; }
    __device__ uint64_t *mbar() const { return g_mbar[warp]; }
    __device__ int warp_elems() const { return 2 * stage_elems() + 2 * TILE1 + TILEI + 32; }
    // the warp regions of the CTA, contiguous: complex scratch of the FFT phases
    __device__ float2 *fft_scratch() const { return reinterpret_cast<float2 *>(sb0 - warp * warp_elems()); }
    __device__ S *red() const { return reinterpret_cast<S *>(g_red); }
    __device__ S *bcast() const { return reinterpret_cast<S *>(g_bcast); }
    __device__ S *gbuf() const { return reinterpret_cast<S *>(g_gbuf); }
    __device__ T *tau() const { return reinterpret_cast<T *>(g_tau); }
    __device__ int tid() const { return threadIdx.x; }
    __device__ int nw() const { return blockDim.x >> 5; }
    __device__ int gw() const { return warp * nblk + bid; }
    __device__ int TW() const { return nblk * nw(); }
    __device__ int off() const { return cx.r4 - cx.r; }
    __device__ int ns() const { return cx.Kp / PC; }

    __device__ Eng(const Ctx<T> &c, const Ctx<T> *maps, int nblk_, int bid_, unsigned char *smem)
        : cx(c), mc(maps), mph(0), wslot(1), nblk(nblk_), bid(bid_), epoch(0), alive(true), tmafail(false), gedge(true),
          fph(0), fpend(0), ffail(false)
    {
        lane = threadIdx.x & 31;
        warp = threadIdx.x >> 5;
        const Layout<T> L(cx.C, cx.K, nw(), cx.wsm, kFFT);
        T *base = reinterpret_cast<T *>(smem);   // 128-byte aligned (checked by the kernel)
        wF = wT = nullptr;
        wsm = base;
        sb0 = base + L.w_elems + warp * L.warp_elems;
        if (lane == 0) {
            mbar_init(&mbar()[0], 1);
            mbar_init(&mbar()[1], 1);
            if (kFFT && warp == 0)
                for (int i = 0; i < 3; ++i) mbar_init(&g_fmbar[i], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }

    // ------------------------------------------------------------ plumbing
    __device__ bool sync()
    {
        if (!alive) return false;
        fence_proxy_async();           // this thread's global writes, for TMA reads after the barrier
        ++epoch;
        const bool tr = cx.trace && bid == 0 && tid() == 0 && (int)epoch <= cx.trace_cap;
        if (tr) cx.trace[2 * (epoch - 1)] = (long long)globaltimer_ns();
        alive = grid_sync(cx.bar, epoch, (unsigned)nblk, &cx.out->status, cx.timeout_ns, &g_sflag);
        if (tr) cx.trace[2 * (epoch - 1) + 1] = (long long)globaltimer_ns();
        return alive;
    }

    // record a failure status (first one wins); callers unwind uniformly
    __device__ void raise(int st) const { atomicCAS(&cx.out->status, ST_OK, st); }

    __device__ long long gstride() const { return (long long)nblk * blockDim.x; }
    __device__ long long gstart() const { return (long long)bid * blockDim.x + tid(); }

    __device__ T *buf(int b) const { return cx.ws + (long long)b * cx.Np; }
    // offset of pixel (c, i, j) inside a buffer
    __device__ int pidx(int c, int i, int j) const { return c * (int)cx.HWp + (i + cx.Gy) * cx.Wp + (j + cx.Gx); }

    // write pixel (c, i, j) of buffer B and its periodic copies in the ghosts.
    // gedge (warp-uniform, set per strip by strip_of) is false when no pixel of
    // the strip lies within a ghost width of an edge: a plain store then.
    // Otherwise a pixel has at most one column copy and one row copy (plus the
    // corner), as ghosts are at most half the image wide, except when the
    // image is narrower than that (multiwrap: every copy in range).
    __device__ void put(T *B, int c, int i, int j, T v) const
    {
        const int o = c * (int)cx.HWp + (i + cx.Gy) * cx.Wp + (j + cx.Gx);
        B[o] = v;
        if (!gedge) return;
        if (cx.multiwrap) {
            const int cb = c * (int)cx.HWp;
            for (int ii = i - ((i + cx.Gy) / cx.H) * cx.H; ii < cx.H + cx.Gy; ii += cx.H)
                for (int jj = j - ((j + cx.Gx) / cx.W) * cx.W; jj < cx.W + cx.Gx; jj += cx.W)
                    B[cb + (ii + cx.Gy) * cx.Wp + (jj + cx.Gx)] = v;
            return;
        }
        const int ox = j < cx.Gx ? cx.W : (j >= cx.W - cx.Gx ? -cx.W : 0);
        const int oy = i < cx.Gy ? cx.H * cx.Wp : (i >= cx.H - cx.Gy ? -cx.H * cx.Wp : 0);
        if (ox) B[o + ox] = v;
        if (oy) B[o + oy] = v;
        if (ox && oy) B[o + ox + oy] = v;
    }

    // The ghost rows that the real-to-complex phases read, for rows i0 ..
    // i0+nr-1 of channel c of B: image row 0 into padded row H and image row
    // H-1 into padded row -1, interior columns only (val(i - i0, j) gives
    // pixel (i, j)).  Those phases stage rows with one halo row on each side
    // and wrap their stencils' columns in shared memory, so no other ghost
    // cell of the buffers they write is ever read (their CG update keeps its
    // ghost rows at distance 1 from these).
    template <typename V>
    __device__ void halo_rows(T *B, int c, int i0, int nr, V val) const
    {
        const int H = cx.H, W = cx.W;
        T *base = B + c * cx.HWp + cx.Gx;
        if (i0 == 0) {
            T *row = base + (long long)(H + cx.Gy) * cx.Wp;
            for (int j = threadIdx.x; j < W; j += blockDim.x) row[j] = val(0, j);
        }
        if (i0 + nr == H) {
            T *row = base + (long long)(cx.Gy - 1) * cx.Wp;
            for (int j = threadIdx.x; j < W; j += blockDim.x) row[j] = val(nr - 1, j);
        }
    }

    __device__ void strip_of(int s, int &c, int &row0, int &col0)
    {
        const int per = cx.nx * cx.ny;
        c = s / per;
        const int rem = s - c * per;
        const int sy = rem / cx.nx;
        row0 = sy * MR;
        col0 = (rem - sy * cx.nx) * 32;
        gedge = cx.multiwrap || col0 < cx.Gx || col0 + 32 > cx.W - cx.Gx || row0 < cx.Gy || row0 + MR > cx.H - cx.Gy;
    }

    // TMA boxes of buffer b for the strip at (c, row0, col0); lane 0 only.
    // Stage: tile rows trow .. trow+NX-1 (image rows row0 - r + trow ...), BW
    // columns from image column col0 - r4; rows outside the padded image read 0.
    __device__ void box_s(T *dst, int b, int c, int row0, int col0, int trow, uint64_t *mb) const
    {
        tma_load_4d(dst, &mc->map_s, col0 - cx.r4 + cx.Gx, row0 - cx.r + cx.Gy + trow, c, b, mb);
    }
    // halo-1 tile: rows row0-1 .. row0+MR, columns col0-4 .. col0+35 (pitch 40)
    __device__ void box_1(T *dst, int b, int c, int row0, int col0, uint64_t *mb) const
    {
        tma_load_4d(dst, &mc->map_1, col0 - 4 + cx.Gx, row0 - 1 + cx.Gy, c, b, mb);
    }
    // interior: rows row0 .. row0+MR-1, columns col0 .. col0+31 (pitch 32)
    __device__ void box_i(T *dst, int b, int c, int row0, int col0, uint64_t *mb) const
    {
        tma_load_4d(dst, &mc->map_i, col0 + cx.Gx, row0 + cx.Gy, c, b, mb);
    }
    __device__ unsigned bytes_s() const { return (unsigned)(cx.BW * NX * sizeof(T)); }
    __device__ static constexpr unsigned bytes_1() { return (unsigned)(40 * (MR + 2) * sizeof(T)); }
    __device__ static constexpr unsigned bytes_i() { return (unsigned)(32 * MR * sizeof(T)); }
    __device__ T *sb(int i) const { return i ? sb1() : sb0; }

    // wait for the copies on mbar[i]; warp-uniform result.  On a timeout the
    // status is raised and the warp stops its TMA work (tmafail).
    __device__ bool land(int i)
    {
        const unsigned ph = (mph >> i) & 1u;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&mbar()[i], ph, cx.timeout_ns));
        if (!ok) {
            if (lane == 0) raise(ST_TIMEOUT);
            tmafail = true;
            return false;
        }
        mph ^= 1u << i;
        return true;
    }

    // bounded wait for whatever copies a failed warp may still have in flight
    __device__ void drain()
    {
        if (tmafail)
            for (int i = 0; i < 2; ++i) mbar_wait(&mbar()[i], (mph >> i) & 1u, cx.timeout_ns);
        if (ffail) fdrain();
    }
    // bounded wait for the FFT phases' bulk copies still in flight (every thread)
    __device__ void fdrain()
    {
        for (int i = 0; i < 3; ++i)
            if ((fpend >> i) & 1u) {
                mbar_wait(&g_fmbar[i], (fph >> i) & 1u, cx.timeout_ns);
                fph ^= 1u << i;
            }
        fpend = 0;
    }
    // every thread: wait (bounded) for the copies on g_fmbar[i]; CTA-uniform
    // result.  On a timeout the status is raised and the CTA stops issuing
    // (ffail); the next grid barrier then fails everywhere.
    __device__ bool fland(int i)
    {
        const bool ok = __syncthreads_and(mbar_wait(&g_fmbar[i], (fph >> i) & 1u, cx.timeout_ns)) != 0;
        if (!ok) {
            if (tid() == 0) raise(ST_TIMEOUT);
            ffail = true;
            return false;
        }
        fph ^= 1u << i;
        fpend &= ~(1u << i);
        return true;
    }

    // lane 0: expect and issue stage k (buffer k & 1) of image img at tile row
    // trow; extra(mb) issues more boxes (extra_bytes) on the same barrier
    template <typename Extra>
    __device__ void issue(int k, int img, int c, int row0, int col0, int trow, unsigned extra_bytes, Extra extra)
    {
        if (lane == 0) {
            uint64_t *mb = &mbar()[k & 1];
            mbar_expect_tx(mb, bytes_s() + extra_bytes);
            box_s(sb(k & 1), img, c, row0, col0, trow, mb);
            extra(mb);
        }
    }

    // both orientations of kernel b (all channels), column-major per channel:
    // w[c][q][p], p < Kp (rows beyond K are zero).  When they fit (cx.wsm)
    // each CTA keeps them in shared memory; otherwise all CTAs fill the global
    // slot not used by the previous kernel and pass a grid barrier, and the
    // correlation reads them through L1.  Either way the correlation loads
    // them through the same (generic) pointers.
    __device__ void load_weights(const T *b)
    {
        const int K = cx.K, Kp = cx.Kp, KK = K * K, per = Kp * K, n = cx.C * per;
        T *F;
        long long e0, st;
        if (cx.wsm) {
            __syncthreads();           // the previous kernel's readers are done
            F = wsm;
            e0 = tid();
            st = blockDim.x;
        } else {
            wslot ^= 1;
            F = cx.wg + (long long)wslot * 2 * n;
            e0 = gstart();
            st = gstride();
        }
        T *Tt = F + n;
        for (long long e = e0; e < n; e += st) {
            const int c = (int)(e / per), rem = (int)(e - (long long)c * per), q = rem / Kp, p = rem - q * Kp;
            T f = T(0), t = T(0);
            if (p < K) {
                const T *bc = b + (long long)c * KK;
                f = __ldcg(bc + (K - 1 - p) * K + (K - 1 - q));
                t = __ldcg(bc + p * K + q);
            }
            F[e] = f;
            Tt[e] = t;
        }
        wF = F;
        wT = Tt;
        if (cx.wsm) __syncthreads();
        else sync();
        if constexpr (kFFT) spectrum(b);
    }

    __device__ S *partS(int slot) const { return reinterpret_cast<S *>(cx.part) + slot * nblk; }

    // record this CTA's partial in a slot and return the grid total after a
    // barrier; every CTA obtains identical bits
    __device__ S reduce(S mine, int slot)
    {
        const S cta = block_sum<T>(mine, red());
        if (tid() == 0) partS(slot)[bid] = cta;
        if (!sync()) return Sc::zero();
        return grid_total<T>(partS(slot), nblk, gbuf(), bcast());
    }

    // acc += correlation of stage buffer s (kernel rows p0 .. p0+PC-1,
    // kernel columns q0 .. q1-1)
    __device__ void corr_on(const T *s, bool flip, int c, int p0, int q0, int q1, T (&acc)[MR]) const
    {
        const int o = c * cx.Kp * cx.K + p0;
        if (cx.wsm)   // from the shared base itself, so that the loads are known to be shared
            corr_stage<T, MR, PC>(s, cx.BW, wsm + (flip ? 0 : cx.C * cx.Kp * cx.K) + o, q0, q1, cx.Kp, lane + off(), acc);
        else
            corr_stage<T, MR, PC>(s, cx.BW, (flip ? wF : wT) + o, q0, q1, cx.Kp, lane + off(), acc);
    }
    __device__ void corr_on(const T *s, bool flip, int c, int p0, T (&acc)[MR]) const
    {
        corr_on(s, flip, c, p0, 0, cx.K, acc);
    }

    // ------------------------------------------------------------ FFT path
    // Row transforms of batches of cx.frb consecutive image rows (the C*H
    // rows, channel-major) and column transforms of blocks of cx.fcb columns,
    // in the CTA's scratch (the warp regions).  Frequencies are kept in
    // bit-reversed order along both axes (forward DIF, inverse DIT), in cx.fz
    // and in the spectrum cx.fs alike.  Copies between global memory and the
    // scratch go through registers FU elements per thread at a time, so that
    // a thread has that many global loads in flight (the scratch is reached
    // through a generic pointer, so loads would otherwise wait for the
    // preceding stores).
    static constexpr int FU = 8;
    enum { FM_B = 0, FM_BT = 1, FM_GRAM = 2 };   // what multiplies the image's spectrum

    // for e = tid, tid + blockDim, ... < n: v = ld(e), then st(e, v), FU at a
    // time (the loads past n re-read element n - 1 and are discarded)
    template <typename Ld, typename St>
    __device__ void fft_copy(int n, Ld ld, St st)
    {
        const int bd = blockDim.x;
        for (int e0 = tid(); e0 < n; e0 += FU * bd) {
            float2 v[FU];
#pragma unroll
            for (int u = 0; u < FU; ++u) v[u] = ld(min(e0 + u * bd, n - 1));
#pragma unroll
            for (int u = 0; u < FU; ++u)
                if (e0 + u * bd < n) st(e0 + u * bd, v[u]);
        }
    }

    // forward row transforms of rows r0 .. r0+frb-1 of val(c, i, j) into cx.fz
    template <typename Val>
    __device__ void fft_rows_fwd(int r0, Val val)
    {
        float2 *a = fft_scratch();
        const int lh = cx.flogH, W = cx.W, lw = cx.flogW, RB = cx.frb;
        fft_copy(RB * W,
                 [=](int e) {
                     const int ri = r0 + (e >> lw);
                     return make_float2(val(ri >> lh, ri & ((1 << lh) - 1), e & (W - 1)), 0.f);
                 },
                 [=](int e, float2 v) { a[fslot(e >> lw, e & (W - 1), RB)] = v; });
        __syncthreads();
        fft_stages<true>(a, W, lw, RB, cx.ftwW, false);
        float2 *z = cx.fz + (long long)r0 * W;
        fft_copy(RB * W, [=](int e) { return a[fslot(e >> lw, e & (W - 1), RB)]; },
                 [=](int e, float2 v) { z[e] = v; });
        __syncthreads();
    }

    // Kernel spectrum F(k) of kernel bk (C x K x K) into cx.fs: the kernel
    // image k(u, v) = bk[u + r, v + r] at (u mod H, v mod W) (taps that wrap
    // onto the same pixel add up), then the 2-D forward transform.
    __device__ bool spectrum(const T *bk)
    {
        if constexpr (kFFT) {
            if (!sync()) return false;            // no CTA still reads the scratch image
            const int H = cx.H, W = cx.W, K = cx.K, r = cx.r;
            for (int r0 = bid * cx.frb; r0 < cx.C * H; r0 += nblk * cx.frb)
                fft_rows_fwd(r0, [=](int c, int i, int j) {
                    const T *bc = bk + (long long)c * K * K;
                    float v = 0.f;
                    // kernel rows and columns landing on (i, j): p = i + r (mod H), q = j + r (mod W)
                    for (int pp = (i + r) % H; pp < K; pp += H)
                        for (int qq = (j + r) % W; qq < K; qq += W) v += __ldcg(bc + pp * K + qq);
                    return v;
                });
            if (!sync()) return false;
            fft_columns(FM_B, CM_STORE, cx.fs);
            if (!cx.fr2c) return sync();
            if (!sync()) return false;
            gram_symbol();
            return sync();
        } else {
            return false;
        }
    }

    // Column transforms over cx.fz (or, for CM_INV, over src) in blocks of
    // cx.fcb columns.  After the forward transform of the block:
    //   CM_CONV   times the spectrum (FM_B), its conjugate (FM_BT) or its squared
    //             modulus (FM_GRAM, the operator B^T B), inverse, back into cx.fz;
    //   CM_STORE  dst = the transform;
    //   CM_XSTORE dst = src . conj(transform);  CM_XADD dst += src . conj(transform)
    //             (cross-correlation spectra; dst may be src);
    //   CM_INV    (no forward transform) the inverse of src's columns into cx.fz.
    enum { CM_CONV = 0, CM_STORE = 1, CM_XSTORE = 2, CM_XADD = 3, CM_INV = 4 };
    __device__ void fft_columns(int fm, int cm = CM_CONV, float2 *dst = nullptr, const float2 *src = nullptr)
    {
        float2 *a = fft_scratch();
        const int H = cx.H, W = cx.W, lh = cx.flogH, CB = cx.fcb, lcb = __ffs(CB) - 1, nbc = W / CB;
        const int n = H * CB, bd = blockDim.x;
        for (int cbi = bid; cbi < cx.C * nbc; cbi += nblk) {
            const int c = cbi / nbc, j0 = (cbi - c * nbc) * CB;
            const long long o = (long long)c * H * W + j0;
            auto gidx = [=](int e) { return (long long)(e >> lcb) * W + (e & (CB - 1)); };
            auto sidx = [=](int e) { return fslot(e & (CB - 1), e >> lcb, CB); };
            const float2 *zc = (cm == CM_INV ? src : cx.fz) + o;
            fft_copy(n, [=](int e) { return __ldcg(zc + gidx(e)); }, [=](int e, float2 v) { a[sidx(e)] = v; });
            __syncthreads();
            if (cm != CM_INV) fft_stages<true>(a, H, lh, CB, cx.ftwH, false);
            if (cm == CM_STORE) {
                float2 *dc = dst + o;
                fft_copy(n, [=](int e) { return a[sidx(e)]; }, [=](int e, float2 v) { dc[gidx(e)] = v; });
                __syncthreads();
                continue;
            }
            if (cm == CM_XSTORE || cm == CM_XADD) {
                float2 *dc = dst + o;
                const float2 *sc = src + o;
                for (int e0 = tid(); e0 < n; e0 += FU * bd) {
                    float2 sv[FU], dv[FU];
#pragma unroll
                    for (int u = 0; u < FU; ++u) {
                        const long long g = gidx(min(e0 + u * bd, n - 1));
                        sv[u] = __ldcg(sc + g);
                        dv[u] = cm == CM_XADD ? __ldcg(dc + g) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < FU; ++u) {
                        const int e = e0 + u * bd;
                        if (e < n) {
                            const float2 t = a[sidx(e)];
                            const float2 pr = cmul(sv[u], make_float2(t.x, -t.y));
                            dc[gidx(e)] = make_float2(dv[u].x + pr.x, dv[u].y + pr.y);
                        }
                    }
                }
                __syncthreads();
                continue;
            }
            if (cm == CM_CONV) {
                const float2 *sc = cx.fs + o;
                const float sgn = fm == FM_B ? 1.f : -1.f;
                fft_copy(n, [=](int e) { return __ldcg(sc + gidx(e)); },
                         [=](int e, float2 sp) {
                             const int sl = sidx(e);
                             if (fm == FM_GRAM) {
                                 const float m2 = fmaf(sp.x, sp.x, sp.y * sp.y);
                                 a[sl] = make_float2(a[sl].x * m2, a[sl].y * m2);
                             } else {
                                 a[sl] = cmul(a[sl], make_float2(sp.x, sgn * sp.y));
                             }
                         });
                __syncthreads();
            }
            fft_stages<false>(a, H, lh, CB, cx.ftwH, true);
            float2 *zw = cx.fz + o;
            fft_copy(n, [=](int e) { return a[sidx(e)]; }, [=](int e, float2 v) { zw[gidx(e)] = v; });
            __syncthreads();
        }
    }

    // forward row transforms of padded buffer img into cx.fz (less the
    // per-channel offset off[c] when off is given)
    __device__ void fft_rows_img(int img, const double *off = nullptr)
    {
        const T *src = buf(img);
        const long long HWp = cx.HWp;
        const int Wp = cx.Wp, Gy = cx.Gy, Gx = cx.Gx;
        for (int r0 = bid * cx.frb; r0 < cx.C * cx.H; r0 += nblk * cx.frb)
            fft_rows_fwd(r0, [=](int c, int i, int j) {
                const float v = (float)__ldcg(src + c * HWp + (long long)(i + Gy) * Wp + Gx + j);
                return off ? (float)((double)v - off[c]) : v;
            });
    }

    // per-channel sums of the image pixels of buffers b[0..3] into
    // out[4 c + k] (every CTA obtains the same values: per-CTA partials in
    // FP64, then a fixed-order total); needs 4 C doubles at out and
    // nblk x 4 C doubles of cx.zpart.  Ends with a grid barrier.
    __device__ bool chan_sums(const int (&b)[4], double *out)
    {
        const int C = cx.C, W = cx.W;
        double *part = cx.zpart;
        for (int c = 0; c < C; ++c) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int i = bid; i < cx.H; i += nblk)                  // rows dealt to CTAs
                for (int j = tid(); j < W; j += blockDim.x)
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[k] += (double)__ldcg(buf(b[k]) + pidx(c, i, j));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double sk = block_sum_d(acc[k], g_redd);
                if (tid() == 0) part[(long long)bid * 4 * C + 4 * c + k] = sk;
            }
        }
        if (!sync()) return false;
        for (int e = tid(); e < 4 * C; e += blockDim.x) {
            double t = 0.0;
            for (int q = 0; q < nblk; ++q) t += __ldcg(part + (long long)q * 4 * C + e);
            out[e] = t;
        }
        __syncthreads();
        return true;
    }

    // inverse row transforms of cx.fz, real part / (H W) into out (dense)
    __device__ void fft_rows_inv(T *out)
    {
        float2 *a = fft_scratch();
        const int H = cx.H, W = cx.W, lw = cx.flogW, RB = cx.frb;
        const float scale = 1.f / ((float)H * (float)W);
        for (int r0 = bid * RB; r0 < cx.C * H; r0 += nblk * RB) {
            const float2 *z = cx.fz + (long long)r0 * W;
            fft_copy(RB * W, [=](int e) { return __ldcg(z + e); },
                     [=](int e, float2 v) { a[fslot(e >> lw, e & (W - 1), RB)] = v; });
            __syncthreads();
            fft_stages<false>(a, W, lw, RB, cx.ftwW, true);
            T *o = out + (long long)r0 * W;
            fft_copy(RB * W, [=](int e) { return a[fslot(e >> lw, e & (W - 1), RB)]; },
                     [=](int e, float2 v) { o[e] = v.x * scale; });
            __syncthreads();
        }
    }

    // B img (FM_B), B^T img (FM_BT) or B^T B img (FM_GRAM) for buffer img
    // through the 2-D transform with the spectrum of the loaded kernel, into
    // dst (dense; cx.fout when null); ends with a grid barrier.
    __device__ bool fft_conv(int fm, int img, T *dst = nullptr)
    {
        if constexpr (kFFT) {
            fft_rows_img(img);
            if (!sync()) return false;
            fft_columns(fm);
            if (!sync()) return false;
            fft_rows_inv(dst ? dst : cx.fout);
            return sync();
        } else {
            return false;
        }
    }

    // FFT path of the kernel-gradient correlation: with U = B v and
    // V = B x - y in their buffers, out[c, p, q] = sum_n U[n] x[n - d] +
    // V[n] v[n - d] at the lag d = (p - r, q - r) is the inverse transform of
    // F(U) conj(F(x)) + F(V) conj(F(v)), read at d (mod H, W).  Into cx.fout.
    //
    // x and v enter the transforms less their channel means m_x, m_v (the
    // products' zero-frequency terms then vanish, and with them the largest
    // source of rounding spread over every lag); the means come back as
    // m_x sum U + m_v sum V, added exactly to every lag of the channel:
    // cross_off()[c] after the call.
    __device__ double *cross_off() const { return g_xoff; }
    __device__ bool fft_cross(int bx, int bv)
    {
        if constexpr (kFFT) {
            const int steps[4] = {B_U, bx, B_V, bv};
            const int modes[4] = {CM_STORE, CM_XSTORE, CM_STORE, CM_XADD};
            float2 *dsts[4] = {cx.fs, cx.fs, cx.fy, cx.fs};
            const float2 *srcs[4] = {nullptr, cx.fs, nullptr, cx.fy};
            const int sb[4] = {B_U, bx, B_V, bv};
            if (!chan_sums(sb, g_csum)) return false;
            const double n = (double)cx.HW;
            for (int c = tid(); c < cx.C; c += blockDim.x) {
                g_mx[c] = g_csum[4 * c + 1] / n;
                g_mv[c] = g_csum[4 * c + 3] / n;
                g_xoff[c] = g_mx[c] * g_csum[4 * c] + g_mv[c] * g_csum[4 * c + 2];
            }
            __syncthreads();
            for (int k = 0; k < 4; ++k) {
                fft_rows_img(steps[k], k == 1 ? g_mx : (k == 3 ? g_mv : nullptr));
                if (!sync()) return false;
                fft_columns(FM_B, modes[k], dsts[k], srcs[k]);
                if (!sync()) return false;
            }
            fft_columns(FM_B, CM_INV, nullptr, cx.fs);
            if (!sync()) return false;
            fft_rows_inv(cx.fout);
            return sync();
        } else {
            return false;
        }
    }

    // ------------------------------------------------ FFT path, real-to-complex pipeline
    // The FISTA iteration of the lower solve in two grid phases instead of the
    // complex pipeline's four.  The image is real, so its 2-D DFT is kept for
    // the column frequencies nu = 0 .. W/2 only: fzh[c][i][nu] (nu < W/2) and
    // fzn[c][i] (nu = W/2) hold the row DFTs X_i[nu] of the rows i in natural
    // order.
    //   row phase:    rows 2m and 2m+1 of a channel are transformed together
    //                 as z = u_2m + i u_2m+1; Hermitian symmetry separates
    //                 them, X_2m[nu] = (Z[nu] + conj Z[-nu]) / 2 and
    //                 X_2m+1[nu] = (Z[nu] - conj Z[-nu]) / (2i), and packs them
    //                 back for the inverse.  In the FISTA mode the inverse row
    //                 transform of (B^T B y_k)'s half spectra, the gradient
    //                 G = B^T B y_k - B^T y_delta + alpha grad J(y_k), the
    //                 updates x_{k+1}, y_{k+1} and the forward row transform of
    //                 y_{k+1} happen in one visit of the rows (B^T y_delta is
    //                 an image, computed once per solve).
    //   column phase: per block of fcb2 half-spectrum columns, the forward
    //                 column transform, the product with |F(k)|^2 (the symbol
    //                 of B^T B, real), the inverse column transform.
    // Operands are staged into shared memory with cp.async, double buffered
    // where they fit, so that the next task's loads run under the current
    // task's transforms.
    enum { RF_FWD = 0, RF_FISTA = 1, RF_CGP = 2, RF_HESS = 3 };

    // row phase: fnst half-spectrum stages, the image-row buffer, the work area
    __device__ float *rstage(int k) const { return reinterpret_cast<float *>(fft_scratch()) + k * cx.fstage; }
    __device__ float *rrows() const { return rstage(cx.fnst); }
    __device__ float2 *rwork() const { return reinterpret_cast<float2 *>(rrows() + cx.frows); }
    // column phase: fncs stages of the half spectra
    __device__ float2 *cstage(int k) const { return fft_scratch() + k * cx.fcstage; }

    // |F(k)|^2 at the half-spectrum columns from the complex spectrum cx.fs
    // (bit-reversed along both axes): fsh[((c*nb + blk)*H + mu)*fcb2 + k] at
    // column nu = blk*fcb2 + k, fsn[c*H + mu] at nu = W/2 (bit-reversed row
    // position mu, the order of the column phase's forward transform)
    __device__ void gram_symbol()
    {
        const int H = cx.H, W = cx.W, W2 = W / 2, CB = cx.fcb2, nb = W2 / CB, lw = cx.flogW;
        const long long n = (long long)cx.C * H * (W2 + 1);
        for (long long e = gstart(); e < n; e += gstride()) {
            const int c = (int)(e / ((long long)H * (W2 + 1)));
            const int rem = (int)(e - (long long)c * H * (W2 + 1)), mu = rem / (W2 + 1), nu = rem - mu * (W2 + 1);
            const int nupos = (int)(__brev((unsigned)nu) >> (32 - lw)) & (W - 1);
            const float2 f = __ldcg(cx.fs + ((long long)c * H + mu) * W + nupos);
            const float m2 = fmaf(f.x, f.x, f.y * f.y);
            if (nu < W2) {
                const int blk = nu / CB, k = nu - blk * CB;
                const long long o = (((long long)c * nb + blk) * H + mu) * CB + k;
                cx.fsh[o] = m2;
            } else {
                cx.fsn[(long long)c * H + mu] = m2;
            }
        }
    }

    // Staged half spectra: row r of a task at r * spitch() + sidx(nu) (float2;
    // two padding slots after every 32, against the bank conflicts of the
    // bit-reversed reads of the first inverse pass; pairs stay 16-byte aligned)
    __device__ int spitch() const { const int W2 = cx.W / 2; return W2 + 2 * (W2 >> 5); }
    __device__ static int sidx(int nu) { return nu + 2 * (nu >> 5); }
    __device__ int brevw(int v) const { return (int)(__brev((unsigned)v) >> (32 - cx.flogW)) & (cx.W - 1); }

    // copies of row task t (rows i0 .. i0+2frp-1 of channel c): its half
    // spectra into stage st (16-byte cp.async, one group), and, by bulk
    // copies on g_fmbar[2] (warp 0; called by every thread), the image rows
    // i0-1 .. i0+2frp of buffer b1 followed by those of b2 (RF_HESS: again
    // with the halo rows; RF_FISTA: the task's rows only, then those of
    // c = B^T y_delta) into the row buffer.  Shared memory that generic code
    // used must be released to the async proxy (fence_proxy_async_smem and a
    // CTA barrier) before the bulk copies are issued.
    __device__ void rtask_spc(int t, float *st)
    {
        const int W2 = cx.W / 2, RP = cx.frp, tpc = cx.H / (2 * RP), bd = blockDim.x;
        const int c = t / tpc, i0 = (t - c * tpc) * 2 * RP;
        float2 *sp = reinterpret_cast<float2 *>(st);
        const float2 *z = cx.fzh + ((long long)c * cx.H + i0) * W2;
        const int hq = W2 >> 1, spp = spitch();
        for (int e = tid(); e < 2 * RP * hq; e += bd) {
            const int r = e / hq, k2 = 2 * (e - r * hq);
            cp_async16(sp + r * spp + sidx(k2), z + (long long)r * W2 + k2);
        }
        cp_async_commit();
    }
    __device__ void rtask_rows(int t, int mode, int b1, int b2)
    {
        fpend |= 4u;
        if (warp != 0) return;
        const int W = cx.W, RP = cx.frp, tpc = cx.H / (2 * RP);
        const int c = t / tpc, i0 = (t - c * tpc) * 2 * RP;
        // blocks of padded rows: n1 of b1 from r1, n2 of b2 from r2 (after the
        // first block's 2 RP + 2 rows in the RF_FISTA / RF_HESS layout, after
        // its 2 RP rows otherwise); RF_FISTA adds the 2 RP rows of c
        const bool halo = mode == RF_FISTA || mode == RF_HESS;
        const int n1 = halo ? 2 * RP + 2 : 2 * RP, r1 = halo ? i0 - 1 : i0;
        const int n2 = mode == RF_HESS ? 2 * RP + 2 : (mode == RF_FWD || b2 < 0 ? 0 : 2 * RP);
        const int r2 = mode == RF_HESS ? i0 - 1 : i0, o2 = halo ? 2 * RP + 2 : 2 * RP;
        const int nc = mode == RF_FISTA ? 2 * RP : 0;
        uint64_t *mb = &g_fmbar[2];
        if (lane == 0) mbar_expect_tx(mb, (unsigned)((n1 + n2 + nc) * W) * 4u);
        __syncwarp();
        float *rw = rrows();
        for (int q = lane; q < n1 + n2; q += 32) {      // one bulk copy per padded row (its interior)
            const bool first = q < n1;
            const int row = first ? r1 + q : r2 + (q - n1);
            const T *src = buf(first ? b1 : b2) + c * cx.HWp + (long long)(row + cx.Gy) * cx.Wp + cx.Gx;
            bulk_load(rw + (first ? q : o2 + (q - n1)) * W, src, (unsigned)W * 4u, mb);
        }
        // RF_FISTA: rows i0 .. i0+2frp-1 of c = B^T y_delta (dense: one copy)
        if (nc && lane == 0)
            bulk_load(rw + (4 * RP + 2) * W, cx.fc + ((long long)c * cx.H + i0) * W, (unsigned)(nc * W) * 4u, mb);
    }

    // The row phase over all row tasks.  The inverse row transform starts from
    // the staged half spectra (packing rows 2s, 2s+1 as Z = Y_a + i Y_b with
    // Y[-nu] = conj Y[nu]) and leaves the rows in the work area in natural
    // order; the per-pixel step reads them there (RF_HESS: in the last
    // inverse pass's stores), and the forward transform starts from the
    // values it writes back:
    //   RF_FWD:   forward row DFTs of buffer b1 into fzh / fzn.
    //   RF_FISTA: G = B^T B y_k - B^T y_delta + alpha grad J(y_k), y_k in b1,
    //             x_k in b2, B^T y_delta in cx.fc; x_{k+1} = y_k - tau_c G into bo1, y_{k+1} =
    //             x_{k+1} + sc (x_{k+1} - x_k) into bo2 (with its halo rows);
    //             forward row DFTs of y_{k+1}; returns sum G^2.
    //   RF_CGP:   p = r + sc p_prev (r in b1, p_prev in b2; p = r when b2 < 0)
    //             into bo1 (with its halo rows); forward row DFTs of p.
    //   RF_HESS:  Hp = B^T B p + alpha D^T(phi''(D x) . D p), p in b1 (with
    //             halo rows), x in b2, into bo1 (with its halo rows); returns sum p Hp.
    __device__ S rows_r2c(int mode, int b1, int b2, int bo1, int bo2, T sc)
    {
        S part = Sc::zero();
        if constexpr (kFFT) {
            const int H = cx.H, W = cx.W, W2 = W / 2, lw = cx.flogW, RP = cx.frp, ps = cx.fpsh;
            const int lrp = __ffs(RP) - 1, np = fft_npass(lw), spp = spitch();
            const int tpc = H / (2 * RP), ntask = cx.C * tpc, bd = blockDim.x;
            const float scale = 1.f / ((float)H * (float)W);
            const T al = cx.alphaT, g = cx.rpT, ig = cx.irpT;
            const T *tauc = tau();
            float2 *wa = rwork();
            T *O1 = bo1 >= 0 ? buf(bo1) : nullptr, *O2 = bo2 >= 0 ? buf(bo2) : nullptr;
            const T *B1 = buf(b1), *B2 = b2 >= 0 ? buf(b2) : nullptr;
            const bool inv = mode == RF_FISTA || mode == RF_HESS;
            gedge = true;                  // every row has pixels whose copies live in the ghosts
            auto slot = [=](int sq, int e) { return fslotp(sq, e, RP, ps); };
            auto ld_wa = [=](int sq, int e, int) { return wa[slot(sq, e)]; };
            auto st_wa = [=](int sq, int e, int, float2 v) { wa[slot(sq, e)] = v; };
            auto nomid = [](int, int, int, auto &) {};
            int u = 0;
            // copies, double buffered: the next task's half spectra run under
            // this whole task, its image rows under this task's forward passes
            // (issued once the row buffer is free).  Single buffered: the
            // task's own spectrum, then its rows, at the task's start.  Either
            // way the groups complete in the order spectrum(t), rows(t), ...
            const bool dbl = cx.fnst > 1;
            fence_proxy_async_smem();      // earlier phases' use of the scratch, before the copies into it
            __syncthreads();
            if (dbl && bid < ntask) {
                if (inv) rtask_spc(bid, rstage(0));
                rtask_rows(bid, mode, b1, b2);
            }
            for (int t = bid; t < ntask && !ffail; t += nblk, ++u) {
                const int c = t / tpc, i0 = (t - c * tpc) * 2 * RP;
                const bool edge = i0 == 0 || i0 + 2 * RP == H;   // the task writes halo rows
                float *st = rstage(dbl ? (u & 1) : 0);
                const bool nxt = dbl && t + nblk < ntask;
                if (!dbl) {
                    if (inv) rtask_spc(t, st);
                    rtask_rows(t, mode, b1, b2);
                }
                if (inv) {
                    if (nxt) rtask_spc(t + nblk, rstage((u + 1) & 1));
                    if (nxt) cp_async_wait<1>();
                    else cp_async_wait<0>();
                }
                __syncthreads();
                const float2 *sp = reinterpret_cast<const float2 *>(st);
                const float *rw = rrows();                          // rows i0-1 .. i0+2RP of b1, then b2's
                auto rows_landed = [&]() { return fland(2); };
                const float2 *zn = cx.fzn + (long long)c * H + i0;
                // the packed spectrum at bit-reversed position e (first inverse pass)
                auto ld_pack = [=](int sq, int e, int) {
                    const int nu = brevw(e);
                    const float2 *ra = sp + (2 * sq) * spp, *rb = ra + spp;
                    float2 ya, yv;
                    if (nu < W2) {
                        ya = ra[sidx(nu)];
                        yv = rb[sidx(nu)];
                    } else if (nu == W2) {
                        ya = __ldcg(zn + 2 * sq);
                        yv = __ldcg(zn + 2 * sq + 1);
                    } else {
                        const int mq = W - nu;
                        ya = ra[sidx(mq)];
                        yv = rb[sidx(mq)];
                        ya.y = -ya.y;
                        yv.y = -yv.y;
                    }
                    return make_float2(ya.x - yv.y, ya.y + yv.x);
                };
                auto lpass = [&](int i) { return fft_pass_len(lw, i); };
                auto spass = [&](int i) { return fft_pass_s0(lw, i); };
                if (mode == RF_FISTA) {
                    const T tc = tauc[c];
                    const float *xk = rw + (2 * RP + 2) * W;          // x_k, the task's rows
                    const float *cr = rw + (4 * RP + 2) * W;          // c = B^T y_delta, the task's rows
                    for (int i = 0; i < np; ++i) {
                        if (i == 0) fft_pass_n<1>(lpass(i), W, RP, lrp, cx.ftwW, spass(i), ld_pack, nomid, st_wa);
                        else fft_pass_n<1>(lpass(i), W, RP, lrp, cx.ftwW, spass(i), ld_wa, nomid, st_wa);
                        __syncthreads();
                    }
                    if (!rows_landed()) break;
                    // the per-pixel step in natural order, four consecutive
                    // pixels of both rows of a pair per thread: B^T B y_k from
                    // the inverse, - B^T y_delta, + alpha grad J(y_k);
                    // x_{k+1}, y_{k+1} to global memory (interior, 16-byte
                    // stores); y_{k+1} back into the work area for the forward
                    // transform
                    auto pixels = [&](auto regc) {
                        constexpr int REG = decltype(regc)::value;
                        const int lq = lw - 2, q4 = W >> 2;
                        for (int e = tid(); e < RP * q4; e += bd) {
                            const int sq = e >> lq, j0 = (e & (q4 - 1)) << 2;
                            float2 z[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) z[q] = wa[slot(sq, j0 + q)];
                            float yo[2][4];
                            T gs = T(0);       // this thread's share of ||G||^2 (FP32, then float-float)
#pragma unroll
                            for (int pp = 0; pp < 2; ++pp) {
                                const int r = 2 * sq + pp;
                                const float *ym = rw + (r + 1) * W;
                                const float4 yc4 = *reinterpret_cast<const float4 *>(ym + j0);
                                const float4 yu4 = *reinterpret_cast<const float4 *>(ym - W + j0);
                                const float4 yd4 = *reinterpret_cast<const float4 *>(ym + W + j0);
                                const float4 xk4 = *reinterpret_cast<const float4 *>(xk + r * W + j0);
                                const float4 c4 = *reinterpret_cast<const float4 *>(cr + r * W + j0);
                                const float ys[6] = {ym[(j0 - 1) & (W - 1)], yc4.x, yc4.y, yc4.z, yc4.w,
                                                     ym[(j0 + 4) & (W - 1)]};
                                const float yu[4] = {yu4.x, yu4.y, yu4.z, yu4.w};
                                const float yd[4] = {yd4.x, yd4.y, yd4.z, yd4.w};
                                const float xq[4] = {xk4.x, xk4.y, xk4.z, xk4.w};
                                const float cq[4] = {c4.x, c4.y, c4.z, c4.w};
                                float xo[4];
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const T yc = ys[q + 1];
                                    const T tv = dphi<T>(REG, yc - ys[q], g, ig) - dphi<T>(REG, ys[q + 2] - yc, g, ig) +
                                                 dphi<T>(REG, yc - yu[q], g, ig) - dphi<T>(REG, yd[q] - yc, g, ig);
                                    const T gr = (pp ? z[q].y : z[q].x) * scale - cq[q] + al * tv;
                                    const T xnv = yc - tc * gr;
                                    xo[q] = xnv;
                                    yo[pp][q] = xnv + sc * (xnv - xq[q]);
                                    gs += gr * gr;
                                }
                                const int o = pidx(c, i0 + r, j0);
                                *reinterpret_cast<float4 *>(O1 + o) = make_float4(xo[0], xo[1], xo[2], xo[3]);
                                *reinterpret_cast<float4 *>(O2 + o) =
                                    make_float4(yo[pp][0], yo[pp][1], yo[pp][2], yo[pp][3]);
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) wa[slot(sq, j0 + q)] = make_float2(yo[0][q], yo[1][q]);
                            part = Sc::addv(part, gs);
                        }
                    };
                    if (cx.reg == 0) pixels(std::integral_constant<int, 0>());
                    else if (cx.reg == 1) pixels(std::integral_constant<int, 1>());
                    else pixels(std::integral_constant<int, 2>());
                    fence_proxy_async_smem();  // the row buffer's reads, before its refill
                    __syncthreads();
                    halo_rows(O2, c, i0, 2 * RP, [&](int r, int j) {
                        const float2 z = wa[slot(r >> 1, j)];
                        return (r & 1) ? z.y : z.x;
                    });
                    // the row buffer is free: the next task's rows load under
                    // the forward passes
                    if (nxt) rtask_rows(t + nblk, mode, b1, b2);
                    if (edge) __syncthreads();     // the halo rows have read the work area
                    fft_pass_n<0>(lpass(np - 1), W, RP, lrp, cx.ftwW, spass(np - 1), ld_wa, nomid, st_wa);
                    __syncthreads();
                } else if (mode == RF_HESS) {
                    for (int i = 0; i < np; ++i) {
                        if (i == 0) fft_pass_n<1>(lpass(i), W, RP, lrp, cx.ftwW, spass(i), ld_pack, nomid, st_wa);
                        else fft_pass_n<1>(lpass(i), W, RP, lrp, cx.ftwW, spass(i), ld_wa, nomid, st_wa);
                        __syncthreads();
                    }
                    if (!rows_landed()) break;
                    // the per-pixel step, four consecutive pixels of both rows
                    // of a pair per thread: H p = B^T B p (from the inverse) +
                    // alpha D^T(phi''(D x) . D p) to global memory (interior,
                    // 16-byte stores; the work area keeps it for the ghost
                    // copies), <p, H p>
                    auto pixels = [&](auto regc) {
                        constexpr int REG = decltype(regc)::value;
                        const int lq = lw - 2, q4 = W >> 2;
                        for (int e = tid(); e < RP * q4; e += bd) {
                            const int sq = e >> lq, j0 = (e & (q4 - 1)) << 2;
                            float2 z[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) z[q] = wa[slot(sq, j0 + q)];
                            float ho[2][4];
                            T ps = T(0);       // this thread's share of <p, H p> (FP32, then float-float)
#pragma unroll
                            for (int pp = 0; pp < 2; ++pp) {
                                const int r = 2 * sq + pp;
                                const float *pm = rw + (r + 1) * W, *xm = pm + (2 * RP + 2) * W;
                                const float4 pc4 = *reinterpret_cast<const float4 *>(pm + j0);
                                const float4 pu4 = *reinterpret_cast<const float4 *>(pm - W + j0);
                                const float4 pd4 = *reinterpret_cast<const float4 *>(pm + W + j0);
                                const float4 xc4 = *reinterpret_cast<const float4 *>(xm + j0);
                                const float4 xu4 = *reinterpret_cast<const float4 *>(xm - W + j0);
                                const float4 xd4 = *reinterpret_cast<const float4 *>(xm + W + j0);
                                const float ps6[6] = {pm[(j0 - 1) & (W - 1)], pc4.x, pc4.y, pc4.z, pc4.w,
                                                      pm[(j0 + 4) & (W - 1)]};
                                const float xs6[6] = {xm[(j0 - 1) & (W - 1)], xc4.x, xc4.y, xc4.z, xc4.w,
                                                      xm[(j0 + 4) & (W - 1)]};
                                const float pu[4] = {pu4.x, pu4.y, pu4.z, pu4.w}, pd[4] = {pd4.x, pd4.y, pd4.z, pd4.w};
                                const float xu[4] = {xu4.x, xu4.y, xu4.z, xu4.w}, xd[4] = {xd4.x, xd4.y, xd4.z, xd4.w};
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const T xc = xs6[q + 1], pc = ps6[q + 1];
                                    const T wl = ddphi<T>(REG, xc - xs6[q], g, ig);
                                    const T wr = ddphi<T>(REG, xs6[q + 2] - xc, g, ig);
                                    const T wu = ddphi<T>(REG, xc - xu[q], g, ig);
                                    const T wd = ddphi<T>(REG, xd[q] - xc, g, ig);
                                    const T th = wl * (pc - ps6[q]) - wr * (ps6[q + 2] - pc) + wu * (pc - pu[q]) -
                                                 wd * (pd[q] - pc);
                                    const T hv = (pp ? z[q].y : z[q].x) * scale + al * th;
                                    ho[pp][q] = hv;
                                    ps += hv * pc;
                                }
                                *reinterpret_cast<float4 *>(O1 + pidx(c, i0 + r, j0)) =
                                    make_float4(ho[pp][0], ho[pp][1], ho[pp][2], ho[pp][3]);
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) wa[slot(sq, j0 + q)] = make_float2(ho[0][q], ho[1][q]);
                            part = Sc::addv(part, ps);
                        }
                    };
                    if (cx.reg == 0) pixels(std::integral_constant<int, 0>());
                    else if (cx.reg == 1) pixels(std::integral_constant<int, 1>());
                    else pixels(std::integral_constant<int, 2>());
                    fence_proxy_async_smem();  // the row buffer's reads, before its refill
                    __syncthreads();
                    if (nxt) rtask_rows(t + nblk, mode, b1, b2);   // the row buffer is free
                    halo_rows(O1, c, i0, 2 * RP, [&](int r, int j) {
                        const float2 z = wa[slot(r >> 1, j)];
                        return (r & 1) ? z.y : z.x;
                    });
                    continue;                  // no forward transform (the next task starts with a barrier)
                } else {
                    // RF_FWD / RF_CGP: the staged image rows (RF_CGP: p = r + sc
                    // p_prev, to global memory with its halo rows) into the
                    // work area in natural order, four consecutive pixels of
                    // both rows of a pair per thread
                    if (!rows_landed()) break;
                    const int lq = lw - 2, q4 = W >> 2;
                    const bool two = mode == RF_CGP && B2;
                    for (int e = tid(); e < RP * q4; e += bd) {
                        const int sq = e >> lq, j0 = (e & (q4 - 1)) << 2;
                        float4 v[2];
#pragma unroll
                        for (int pp = 0; pp < 2; ++pp) {
                            const int r = 2 * sq + pp;
                            v[pp] = *reinterpret_cast<const float4 *>(rw + r * W + j0);
                            if (two) {
                                const float4 w = *reinterpret_cast<const float4 *>(rw + (2 * RP + r) * W + j0);
                                v[pp] = make_float4(v[pp].x + sc * w.x, v[pp].y + sc * w.y, v[pp].z + sc * w.z,
                                                    v[pp].w + sc * w.w);
                            }
                            if (mode == RF_CGP) *reinterpret_cast<float4 *>(O1 + pidx(c, i0 + r, j0)) = v[pp];
                        }
                        wa[slot(sq, j0)] = make_float2(v[0].x, v[1].x);
                        wa[slot(sq, j0 + 1)] = make_float2(v[0].y, v[1].y);
                        wa[slot(sq, j0 + 2)] = make_float2(v[0].z, v[1].z);
                        wa[slot(sq, j0 + 3)] = make_float2(v[0].w, v[1].w);
                    }
                    fence_proxy_async_smem();  // the row buffer's reads, before its refill
                    __syncthreads();
                    if (nxt) rtask_rows(t + nblk, mode, b1, b2);   // under the forward passes
                    if (mode == RF_CGP) {
                        halo_rows(O1, c, i0, 2 * RP, [&](int r, int j) {
                            const float2 z = wa[slot(r >> 1, j)];
                            return (r & 1) ? z.y : z.x;
                        });
                        if (edge) __syncthreads();   // the halo rows have read the work area
                    }
                    fft_pass_n<0>(lpass(np - 1), W, RP, lrp, cx.ftwW, spass(np - 1), ld_wa, nomid, st_wa);
                    __syncthreads();
                }
                // the remaining forward passes, then separate the two rows'
                // spectra and store nu = 0 .. W/2
                for (int i = np - 2; i >= 0; --i) {
                    fft_pass_n<0>(lpass(i), W, RP, lrp, cx.ftwW, spass(i), ld_wa, nomid, st_wa);
                    __syncthreads();
                }
                float2 *zh = cx.fzh + ((long long)c * H + i0) * W2;
                float2 *znw = cx.fzn + (long long)c * H + i0;
                for (int e = tid(); e < RP * (W2 + 1); e += bd) {
                    const int sq = e / (W2 + 1), nu = e - sq * (W2 + 1);
                    const float2 z1 = wa[slot(sq, brevw(nu))];
                    const float2 z2 = wa[slot(sq, brevw((W - nu) & (W - 1)))];
                    const float2 xa = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
                    const float2 xv = make_float2(0.5f * (z1.y + z2.y), -0.5f * (z1.x - z2.x));
                    if (nu < W2) {
                        zh[(2 * sq) * W2 + nu] = xa;
                        zh[(2 * sq + 1) * W2 + nu] = xv;
                    } else {
                        znw[2 * sq] = xa;
                        znw[2 * sq + 1] = xv;
                    }
                }
                fence_proxy_async_smem();      // the row buffer's reads, before a refill at the next task's start
                __syncthreads();               // the work area is rewritten by the next task
            }
            cp_async_wait<0>();
            if (ffail) fdrain();
            fence_proxy_async_smem();      // before later phases' TMA copies into the same shared memory
        }
        return part;
    }

    // column phase: fncs stages of the half spectra, then as many of the symbol
    __device__ float *csym(int k) const { return reinterpret_cast<float *>(cstage(cx.fncs)) + (long long)k * cx.fcstage; }

    // thread 0: copies of column task t (block blk of channel c, or the
    // column W/2 of channel t - C*nb) into column stage k on g_fmbar[k]: the
    // spectrum dense, element (i, kk) at i * cnt + kk (tensor boxes of fzh;
    // one bulk copy for the column W/2), and the symbol |F(k)|^2 of its
    // columns in the order of fsh / fsn (one bulk copy; the column W/2's
    // only when whole 16-byte units, else the product reads fsn).  Called by
    // every thread (the pending bits stay uniform).
    __device__ void ctask_issue(int t, int k)
    {
        fpend |= 1u << k;
        if (tid() != 0) return;
        const int H = cx.H, W2 = cx.W / 2, CB = cx.fcb2, nb = W2 / CB;
        float2 *a = cstage(k);
        float *sm = csym(k);
        uint64_t *mb = &g_fmbar[k];
        if (t < cx.C * nb) {
            const int c = t / nb, blk = t - c * nb, BR = H < 256 ? H : 256;
            mbar_expect_tx(mb, (unsigned)(H * CB) * 12u);
            for (int r0 = 0; r0 < H; r0 += BR) tma_load_2d(a + r0 * CB, &mc->map_fz, 2 * blk * CB, c * H + r0, mb);
            bulk_load(sm, cx.fsh + ((long long)c * nb + blk) * H * CB, (unsigned)(H * CB) * 4u, mb);
        } else {
            const int c = t - cx.C * nb;
            const bool whole = (H & 3) == 0;
            mbar_expect_tx(mb, (unsigned)H * (whole ? 12u : 8u));
            bulk_load(a, cx.fzn + (long long)c * H, (unsigned)H * 8u, mb);
            if (whole) bulk_load(sm, cx.fsn + (long long)c * H, (unsigned)H * 4u, mb);
        }
    }

    // The column phase over the half spectra in fzh / fzn: forward column
    // transforms, the product with |F(k)|^2 (the symbol of B^T B, staged with
    // the task's spectrum) over the staged spectrum, inverse column
    // transforms, the block back to fzh / fzn by bulk stores.  Double
    // buffered: the next task's copies go out after this task's forward
    // passes, once the store that last read their buffer has read it.
    __device__ void cols_r2c()
    {
        if constexpr (kFFT) {
            const int H = cx.H, lh = cx.flogH, W2 = cx.W / 2, CB = cx.fcb2, nb = W2 / CB;
            const int ntask = cx.C * nb + cx.C, np = fft_npass(lh), bd = blockDim.x;
            const bool dbl = cx.fncs > 1;
            auto nomid = [](int, int, int, auto &) {};
            fence_proxy_async_smem();  // earlier phases' use of the scratch, before the copies into it
            __syncthreads();
            int u = 0;
            if (bid < ntask) ctask_issue(bid, 0);
            for (int t = bid; t < ntask && !ffail; t += nblk, ++u) {
                const int sk = dbl ? (u & 1) : 0;
                if (!fland(sk)) break;
                float2 *a = cstage(sk);
                const float *sm = csym(sk);
                const int tn = t + nblk;
                const bool nyq = t >= cx.C * nb;
                const int cnt = nyq ? 1 : CB, lc = __ffs(cnt) - 1;
                const int c = nyq ? t - cx.C * nb : t / nb, blk = nyq ? 0 : t - c * nb;
                auto ld_a = [=](int sq, int e, int) { return a[e * cnt + sq]; };
                auto st_a = [=](int sq, int e, int, float2 v) { a[e * cnt + sq] = v; };
                auto lpass = [&](int i) { return fft_pass_len(lh, i); };
                auto spass = [&](int i) { return fft_pass_s0(lh, i); };
                for (int i = np - 1; i >= 0; --i) {
                    fft_pass_n<0>(lpass(i), H, cnt, lc, cx.ftwH, spass(i), ld_a, nomid, st_a);
                    __syncthreads();
                }
                if (dbl && tn < ntask) {
                    if (tid() == 0) bulk_wait_read_all();
                    ctask_issue(tn, (u + 1) & 1);
                }
                // element (mu, k) of the task at mu * cnt + k, here and in the symbol
                const float *sg = cx.fsn + (long long)c * H;
                const bool sglob = nyq && (H & 3) != 0;
                for (int e = tid(); e < H * cnt; e += bd) {
                    const float m2 = sglob ? __ldcg(sg + e) : sm[e];
                    a[e] = make_float2(a[e].x * m2, a[e].y * m2);
                }
                __syncthreads();
                for (int i = 0; i < np; ++i) {
                    fft_pass_n<1>(lpass(i), H, cnt, lc, cx.ftwH, spass(i), ld_a, nomid, st_a);
                    __syncthreads();
                }
                fence_proxy_async_smem();  // the block's writes, before the bulk store reads them
                __syncthreads();
                if (tid() == 0) {
                    if (nyq) {
                        bulk_store(cx.fzn + (long long)c * H, a, (unsigned)H * 8u);
                    } else {
                        const int BR = H < 256 ? H : 256;
                        for (int r0 = 0; r0 < H; r0 += BR) tma_store_2d(&mc->map_fz, 2 * blk * CB, c * H + r0, a + r0 * CB);
                    }
                    bulk_commit();
                }
                if (!dbl && tn < ntask) {
                    if (tid() == 0) bulk_wait_read_all();
                    ctask_issue(tn, 0);
                }
            }
            if (ffail) fdrain();
            if (tid() == 0) {
                bulk_wait_all();       // the stores are complete before the grid barrier
                fence_proxy_async();
            }
            fence_proxy_async_smem();
            __syncthreads();
        }
    }

    // FISTA of lower_solve on the real-to-complex pipeline: the same
    // iterates, stopping test and cap as the direct path (the test on
    // ||grad_x h(y_k)|| is read during the column phase of iteration k)
    __device__ int lower_solve_r2c(const T *b, int bin, int bout, double eps, int max_iters, double &gn,
                                   long long &passes)
    {
        load_weights(b);               // spectrum and Gram symbol of b
        compute_tau(b);
        copy_buf(B_X0, B_Y0, bin);
        if (!sync()) return 0;
        // c = B^T y_delta (dense, in cx.fc), once per solve, on the complex pipeline
        if (!fft_conv(FM_BT, B_Y, cx.fc)) return 0;
        rows_r2c(RF_FWD, B_Y0, -1, -1, -1, T(0));
        if (!sync()) return 0;
        cols_r2c();
        if (!sync()) return 0;
        int xp = B_X0, xn = B_X1, yc = B_Y0, yn = B_Y1;
        const S eps2 = Sc::from_double(eps * eps);
        S t = Sc::of(1);
        S tn = next_t(t);
        T th = (T)Sc::to_elem(Sc::div(Sc::addv(t, -1), tn));
        int result = yc, k = 0;
        for (;; ++k) {
            const S part = rows_r2c(RF_FISTA, yc, xp, xn, yn, th);
            const S cta = block_sum<T>(part, red());
            if (tid() == 0) partS(k & 1)[bid] = cta;
            const S t_next = tn;
            const S tn_next = next_t(t_next);
            const T th_next = (T)Sc::to_elem(Sc::div(Sc::addv(t_next, -1), tn_next));
            if (!sync()) return k;
            passes += 1;
            if (k >= max_iters) {
                const S ss = grid_total<T>(partS(k & 1), nblk, gbuf(), bcast());
                if (!Sc::finite(ss)) {
                    if (tid() == 0) raise(ST_NONFINITE);
                    alive = false;
                    return k;
                }
                gn = sqrt(Sc::to_double(ss));
                result = yc;
                break;
            }
            if (warp == 0) grid_issue<T>(partS(k & 1), nblk, gbuf());
            cols_r2c();
            if (warp == 0) {
                const S s = grid_finish<T>(nblk, gbuf());
                if (lane == 0) *bcast() = s;
            }
            __syncthreads();
            const S ss = *bcast();
            __syncthreads();
            if (!Sc::finite(ss)) {
                if (tid() == 0) raise(ST_NONFINITE);
                alive = false;
                return k;
            }
            if (Sc::le(ss, eps2)) {        // y_k passes: x_{k+1}, y_{k+1} are dropped
                gn = sqrt(Sc::to_double(ss));
                result = yc;
                break;
            }
            if (!sync()) return k;
            t = t_next;
            tn = tn_next;
            th = th_next;
            int tmp = xp; xp = xn; xn = tmp;
            tmp = yc; yc = yn; yn = tmp;
        }
        if (result != bout) copy_buf(bout, -1, result);
        return k;
    }

    // pass() on the FFT path: the correlation comes from fft_conv, then the
    // strips run the same epilogue with the same staged operands.
    template <typename Epi>
    __device__ S pass_fft(int fm, int img0, int t1b, int t2b, int fb, Epi epi)
    {
        S part = Sc::zero();
        if (!fft_conv(fm, img0)) return part;
        const unsigned eb = (t1b >= 0 ? bytes_1() : 0u) + (t2b >= 0 ? bytes_1() : 0u) + (fb >= 0 ? bytes_i() : 0u);
        for (int s = gw(); s < cx.nstrips; s += TW()) {
            int c, row0, col0;
            strip_of(s, c, row0, col0);
            if (eb) {
                if (lane == 0) {
                    uint64_t *mb = &mbar()[0];
                    mbar_expect_tx(mb, eb);
                    if (t1b >= 0) box_1(t1(), t1b, c, row0, col0, mb);
                    if (t2b >= 0) box_1(t2(), t2b, c, row0, col0, mb);
                    if (fb >= 0) box_i(tF(), fb, c, row0, col0, mb);
                }
                if (!land(0)) return part;
            }
            T sum = T(0);
            const int gj = col0 + lane;
            const long long cbase = (long long)c * cx.HW;
            T acc[MR];                     // all loads in flight before the epilogue's stores
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int gi = row0 + m;
                acc[m] = (gi < cx.H && gj < cx.W) ? __ldcg(cx.fout + cbase + (long long)gi * cx.W + gj) : T(0);
            }
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int gi = row0 + m;
                if (gi < cx.H && gj < cx.W)
                    sum += epi(c, gi, gj, cbase + (long long)gi * cx.W + gj, m, acc[m], tF()[m * 32 + lane]);
            }
            part = Sc::addv(part, sum);
            __syncwarp();                  // epilogue reads before the next strip's copies
        }
        return part;
    }

    // One convolution pass over all strips.  img0 is staged in stages of NX
    // rows (double-buffered).  With img1 >= 0 each stage holds img0 in sb0 and
    // img1 in sb1() (single-buffered) and prep(stage, c, row0, col0) combines them
    // into sb0 before the correlation.  The halo-1 tiles of t1b / t2b and the
    // interior of fb (epilogue operands, any may be -1) are staged with the
    // first stage.  epi(c, gi, gj, g, m, v, fv) consumes each in-image output v
    // (dense index g, with fv the staged operand) and returns its share of a
    // reduction (element type per strip, reduction scalar across strips).
    template <typename Prep, typename Epi>
    __device__ S pass(bool flip, int img0, int img1, int t1b, int t2b, int fb, Prep prep, Epi epi)
    {
        if constexpr (kFFT) {
            return pass_fft(flip ? FM_B : FM_BT, img0, t1b, t2b, fb, epi);   // img1 is never set here
        }
        S part = Sc::zero();
        if (!alive || tmafail) return part;
        if (lane == 0) fence_proxy_async();
        const bool two = img1 >= 0;
        const unsigned eb = (t1b >= 0 ? bytes_1() : 0u) + (t2b >= 0 ? bytes_1() : 0u) + (fb >= 0 ? bytes_i() : 0u);
        for (int s = gw(); s < cx.nstrips; s += TW()) {
            int c, row0, col0;
            strip_of(s, c, row0, col0);
            auto extra = [&](uint64_t *mb) {
                if (t1b >= 0) box_1(t1(), t1b, c, row0, col0, mb);
                if (t2b >= 0) box_1(t2(), t2b, c, row0, col0, mb);
                if (fb >= 0) box_i(tF(), fb, c, row0, col0, mb);
            };
            T acc[MR];
#pragma unroll
            for (int m = 0; m < MR; ++m) acc[m] = T(0);
            if (!two) {
                issue(0, img0, c, row0, col0, 0, eb, extra);
                for (int st = 0; st < ns(); ++st) {
                    if (!land(st & 1)) return part;
                    if (st + 1 < ns()) issue(st + 1, img0, c, row0, col0, (st + 1) * PC, 0u, [](uint64_t *) {});
                    corr_on(sb(st & 1), flip, c, st * PC, acc);
                    __syncwarp();
                }
            } else {
                for (int st = 0; st < ns(); ++st) {
                    if (lane == 0) {
                        uint64_t *mb = &mbar()[0];
                        mbar_expect_tx(mb, 2 * bytes_s() + (st == 0 ? eb : 0u));
                        box_s(sb0, img0, c, row0, col0, st * PC, mb);
                        box_s(sb1(), img1, c, row0, col0, st * PC, mb);
                        if (st == 0) extra(mb);
                    }
                    if (!land(0)) return part;
                    prep(st, c, row0, col0);
                    __syncwarp();
                    corr_on(sb0, flip, c, st * PC, acc);
                    __syncwarp();
                }
            }
            T sum = T(0);
            const int gj = col0 + lane;
            const long long cbase = (long long)c * cx.HW;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int gi = row0 + m;
                if (gi < cx.H && gj < cx.W)
                    sum += epi(c, gi, gj, cbase + (long long)gi * cx.W + gj, m, acc[m], tF()[m * 32 + lane]);
            }
            part = Sc::addv(part, sum);
            __syncwarp();                  // epilogue reads before the next strip's copies
        }
        return part;
    }

    // TV gradient at strip pixel (m, lane) of a halo-1 tile s (pitch 40,
    // column 0 = image column col0 - 4)
    __device__ T tv_grad(const T *s, int m) const
    {
        const T g = cx.rpT, ig = cx.irpT;
        const int o = (m + 1) * 40 + lane + 4;
        const T yc = s[o];
        return dphi<T>(cx.reg, yc - s[o - 1], g, ig) - dphi<T>(cx.reg, s[o + 1] - yc, g, ig) +
               dphi<T>(cx.reg, yc - s[o - 40], g, ig) - dphi<T>(cx.reg, s[o + 40] - yc, g, ig);
    }

    // D^T(phi''(D x) . D v) at strip pixel (m, lane); x in sx, v in sv (halo 1)
    __device__ T tv_hess(const T *sx, const T *sv, int m) const
    {
        const T g = cx.rpT, ig = cx.irpT;
        const int o = (m + 1) * 40 + lane + 4;
        const T xc = sx[o], vc = sv[o];
        const T wl = ddphi<T>(cx.reg, xc - sx[o - 1], g, ig);
        const T wr = ddphi<T>(cx.reg, sx[o + 1] - xc, g, ig);
        const T wu = ddphi<T>(cx.reg, xc - sx[o - 40], g, ig);
        const T wd = ddphi<T>(cx.reg, sx[o + 40] - xc, g, ig);
        return wl * (vc - sv[o - 1]) - wr * (sv[o + 1] - vc) + wu * (vc - sv[o - 40]) - wd * (sv[o + 40] - vc);
    }

    __device__ T center1(const T *s, int m) const { return s[(m + 1) * 40 + lane + 4]; }

    // ------------------------------------------------------------ import / export
    // dense caller image -> buffer b (with ghosts); a warp per image row
    __device__ void import_dense(const T *src, int b)
    {
        T *B = buf(b);
        gedge = true;                  // rows of any position: ghost copies checked per pixel
        for (int row = gw(); row < cx.C * cx.H; row += TW()) {
            const int c = row / cx.H, i = row - c * cx.H;
            const T *sr = src + (long long)row * cx.W;
            for (int j = lane; j < cx.W; j += 32) put(B, c, i, j, __ldcg(sr + j));
        }
    }

    // buffer b -> dense caller image; a warp per image row
    __device__ void export_dense(int b, T *dst)
    {
        const T *B = buf(b);
        for (int row = gw(); row < cx.C * cx.H; row += TW()) {
            const int c = row / cx.H, i = row - c * cx.H;
            T *dr = dst + (long long)row * cx.W;
            const T *br = B + pidx(c, i, 0);
            for (int j = lane; j < cx.W; j += 32) dr[j] = __ldcg(br + j);
        }
    }

    // dst = src (and dst2 = src) over whole padded buffers, ghosts included
    __device__ void copy_buf(int dst, int dst2, int src)
    {
        const T *Sp = buf(src);
        T *D = buf(dst), *D2 = dst2 >= 0 ? buf(dst2) : nullptr;
        const long long N = cx.Np, st = gstride();
        for (long long base = gstart(); base < N; base += EWB * st) {
            T v[EWB];
#pragma unroll
            for (int u = 0; u < EWB; ++u) {
                const long long i = base + u * st;
                v[u] = i < N ? __ldcg(Sp + i) : T(0);
            }
#pragma unroll
            for (int u = 0; u < EWB; ++u) {
                const long long i = base + u * st;
                if (i < N) {
                    D[i] = v[u];
                    if (D2) D2[i] = v[u];
                }
            }
        }
    }

    // ------------------------------------------------------------ programs
    struct NoPrep {
        __device__ void operator()(int, int, int, int) const {}
    };
    static constexpr NoPrep noprep{};

    // out = B x (flip) or B^T x; x in buffer bx, weights of b loaded
    __device__ void apply(int bx, T *out, bool transpose)
    {
        pass(!transpose, bx, -1, -1, -1, -1, noprep,
             [=](int, int, int, long long g, int, T v, T) { out[g] = v; return T(0); });
    }

    // buffer bu = B x - y (weights of b loaded)
    __device__ void residual(int bx, int bu)
    {
        T *U = buf(bu);
        pass(true, bx, -1, -1, -1, B_Y, noprep,
             [=](int c, int gi, int gj, long long, int, T v, T yv) { put(U, c, gi, gj, v - yv); return T(0); });
    }

    // grad_x h = B^T(B x - y) + alpha grad J(x) into dense out (may be null);
    // its norm into the result record
    __device__ void grad_lower(const T *b, int bx, T *out)
    {
        load_weights(b);
        residual(bx, B_U);
        if (!sync()) return;
        const T al = cx.alphaT;
        const S part = pass(false, B_U, -1, bx, -1, -1, noprep, [=](int, int, int, long long g, int m, T v, T) {
            const T gr = v + al * tv_grad(t1(), m);
            if (out) out[g] = gr;
            return gr * gr;
        });
        const S ss = reduce(part, 0);
        if (alive && tid() == 0 && bid == 0) cx.out->gradnorm = sqrt(Sc::to_double(ss));
    }

    // B^T B v + alpha D^T(phi''(D x) . D v) for x, v in buffers bx, bv: to
    // buffer bo (with ghosts) or, when dense_out is set, to the caller's image.
    // Returns this warp's share of <v, out>.  Weights of b loaded.
    __device__ S hess_vec(int bx, int bv, int bo, T *dense_out)
    {
        if (!gram()) {
            T *U = buf(B_U);
            pass(true, bv, -1, -1, -1, -1, noprep,
                 [=](int c, int gi, int gj, long long, int, T val, T) { put(U, c, gi, gj, val); return T(0); });
            if (!sync()) return Sc::zero();
        }
        return hess_vec_b(bx, bv, bo, dense_out);
    }

    // second half of a Hessian-vector product whose first half (U = B v) is
    // done: out = B^T U + alpha D^T(phi''(D x) . D v); <v, out>
    __device__ S hess_vec_b(int bx, int bv, int bo, T *dense_out)
    {
        const T al = cx.alphaT;
        T *O = buf(bo);
        auto epi = [=](int c, int gi, int gj, long long g, int m, T v, T) {
            const T hv = v + al * tv_hess(t1(), t2(), m);
            if (dense_out) dense_out[g] = hv;
            else put(O, c, gi, gj, hv);
            return hv * center1(t2(), m);
        };
        if (gram()) return pass_fft(FM_GRAM, bv, bx, bv, -1, epi);   // B^T B v in one transform pair
        return pass(false, B_U, -1, bx, bv, -1, noprep, epi);
    }

    // FFT path: B^T B applied through |F(k)|^2 in one forward/inverse pair
    // (the FISTA gradient and the Hessian products)
    __device__ bool gram() const
    {
        if constexpr (kFFT) return true;
        else return false;
    }

    // 1/L_c for FISTA on channel c with kernel b: L_c = ||b_c||_1^2 + 8 alpha sup phi''
    // (the l1 norm in the reduction scalar, the rest in FP64 by one thread)
    __device__ void compute_tau(const T *b)
    {
        const int KK = cx.K * cx.K;
        for (int c = 0; c < cx.C; ++c) {
            S s = Sc::zero();
            for (int e = tid(); e < KK; e += blockDim.x) s = Sc::addv(s, fabs(__ldcg(b + (long long)c * KK + e)));
            const S l1 = block_sum<T>(s, red());
            if (tid() == 0) {
                const double l = Sc::to_double(l1);
                tau()[c] = (T)(1.0 / (l * l + 8.0 * cx.alpha * cx.ddphi_max));
            }
        }
        __syncthreads();
    }

    // t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, the FISTA momentum sequence
    __device__ S next_t(S t) const
    {
        return Sc::mul(Sc::addv(Sc::sqroot(Sc::addv(Sc::mul(Sc::of(4), Sc::mul(t, t)), 1)), 1), Sc::of(0.5));
    }

    // FISTA (Algorithm 1, step 1) from buffer bin (warm start) to buffer bout:
    // returns updates made.  The momentum theta_{k+1} = (t_k - 1)/t_{k+1} does
    // not depend on the data, so pass B writes both x_{k+1} and y_{k+1}.  The
    // stopping test on ||grad_x h(y_k)|| is read one pass late: the partial sums
    // of iteration k are fetched while pass A of iteration k+1 runs, and when
    // the test holds y_k (still in its own buffer) is returned and that pass A
    // is discarded.  bin may equal bout.
    __device__ int lower_solve(const T *b, int bin, int bout, double eps, int max_iters, double &gn,
                               long long &passes)
    {
        if constexpr (kFFT) {
            if (cx.fr2c) return lower_solve_r2c(b, bin, bout, eps, max_iters, gn, passes);
        }
        load_weights(b);
        compute_tau(b);
        copy_buf(B_X0, B_Y0, bin);
        if (!sync()) return 0;
        // FFT path: grad = B^T B y - B^T y_delta + alpha grad J(y), with B^T y_delta once
        if (gram() && !fft_conv(FM_BT, B_Y, cx.fc)) return 0;
        const T *FC = cx.fc;
        int xp = B_X0, xn = B_X1, yc = B_Y0, yn = B_Y1;
        const T al = cx.alphaT;
        const T *tauc = tau();
        int result = -1;
        const S eps2 = Sc::from_double(eps * eps);
        // theta_{k+1} for the first iteration (t_0 = 1); later ones are computed
        // while a barrier is pending
        S t = Sc::of(1);
        S tn = next_t(t);
        T thn = (T)Sc::to_elem(Sc::div(Sc::addv(t, -1), tn));
        bool pending = false;
        int k = 0;
        for (;; ++k) {
            const int ycur = yc;
            if (pending && warp == 0) grid_issue<T>(partS((k - 1) & 1), nblk, gbuf());
            // phase A: U = B y_k - y (not on the FFT path)
            if (!gram()) residual(ycur, B_U);
            if (pending) {
                if (warp == 0) {
                    const S s = grid_finish<T>(nblk, gbuf());
                    if (lane == 0) *bcast() = s;
                }
                __syncthreads();
                const S sprev = *bcast();
                __syncthreads();
                if (!Sc::finite(sprev)) {
                    if (tid() == 0) raise(ST_NONFINITE);
                    alive = false;
                    return k - 1;
                }
                if (Sc::le(sprev, eps2)) {     // y_{k-1} passes: keep it, drop this pass A
                    gn = sqrt(Sc::to_double(sprev));
                    result = yn;
                    --k;
                    break;
                }
            }
            if (!sync()) return k;
            // phase B: G = B^T U + alpha grad J(y_k); x_{k+1} = y_k - tau_c G;
            // y_{k+1} = x_{k+1} + theta_{k+1} (x_{k+1} - x_k); ||G||^2
            T *XN = buf(xn), *YN = buf(yn);
            const T th = thn;
            auto epiB = [=](int c, int gi, int gj, long long, int m, T v, T xpv) {
                const T gr = v + al * tv_grad(t1(), m);
                const T xnv = center1(t1(), m) - tauc[c] * gr;
                XN[pidx(c, gi, gj)] = xnv;     // read back only as an interior operand
                put(YN, c, gi, gj, xnv + th * (xnv - xpv));
                return gr * gr;
            };
            const S part = gram() ? pass_fft(FM_GRAM, ycur, ycur, -1, xp,
                                             [=](int c, int gi, int gj, long long g, int m, T v, T xpv) {
                                                 return epiB(c, gi, gj, g, m, v - __ldcg(FC + g), xpv);
                                             })
                                  : pass(false, B_U, -1, ycur, -1, xp, noprep, epiB);
            const S cta = block_sum<T>(part, red());
            if (tid() == 0) partS(k & 1)[bid] = cta;
            // momentum of the next iteration, before waiting on the barrier
            const S t_next = tn;
            const S tn_next = next_t(t_next);
            const T thn_next = (T)Sc::to_elem(Sc::div(Sc::addv(t_next, -1), tn_next));
            if (!sync()) return k;
            passes += gram() ? 1 : 2;
            if (k >= max_iters) {          // cap: the norm of y_k is needed now
                const S ss = grid_total<T>(partS(k & 1), nblk, gbuf(), bcast());
                if (!Sc::finite(ss)) {
                    if (tid() == 0) raise(ST_NONFINITE);
                    alive = false;
                    return k;
                }
                gn = sqrt(Sc::to_double(ss));
                result = yc;
                break;
            }
            pending = true;
            t = t_next;
            tn = tn_next;
            thn = thn_next;
            int tmp = xp; xp = xn; xn = tmp;
            tmp = yc; yc = yn; yn = tmp;
        }
        if (result != bout) copy_buf(bout, -1, result);
        return k;
    }

    // r(b) = beta (w0 ||d||^2 + ||D_h d||^2 + ||D_v d||^2), d = b - a; every
    // CTA computes it (it is small)
    __device__ T dker(const T *b, long long idx) const { return __ldcg(b + idx) - __ldg(cx.a + idx); }

    __device__ double sobolev(const T *b)
    {
        const int K = cx.K, KK = K * K;
        double s = 0.0;
        for (int e = tid(); e < cx.C * KK; e += blockDim.x) {
            const int c = e / KK, pq = e - c * KK, p = pq / K, q = pq - p * K;
            const long long base = (long long)c * KK;
            const double d = (double)dker(b, base + pq);
            const double dh = q < K - 1 ? (double)dker(b, base + pq + 1) - d : 0.0;
            const double dv = p < K - 1 ? (double)dker(b, base + pq + K) - d : 0.0;
            s += cx.w0 * d * d + dh * dh + dv * dv;
        }
        return cx.beta * block_sum_d(s, g_redd);
    }

    __device__ double grad_sobolev_elem(const T *b, int e) const
    {
        const int K = cx.K, KK = K * K;
        const int c = e / KK, pq = e - c * KK, p = pq / K, q = pq - p * K;
        const long long base = (long long)c * KK;
        const double d = (double)dker(b, base + pq);
        auto at = [&](int pp, int qq) { return (double)dker(b, base + pp * K + qq); };
        const double dh_here = q < K - 1 ? at(p, q + 1) - d : 0.0;
        const double dh_prev = q >= 1 ? d - at(p, q - 1) : 0.0;
        const double dv_here = p < K - 1 ? at(p + 1, q) - d : 0.0;
        const double dv_prev = p >= 1 ? d - at(p - 1, q) : 0.0;
        return 2.0 * cx.beta * (cx.w0 * d + dh_prev - dh_here + dv_prev - dv_here);
    }

    // ell = g(x) + r(b) and ||grad g(x)|| for x in buffer bx; grad g = 2 A^T(A x - y)
    // stored in buffer B_G (with ghosts)
    __device__ void upper_loss(const T *b, int bx, double &loss, double &gxn, long long &passes)
    {
        // r(b) first: b may be rewritten by other CTAs right after the last
        // barrier of this function (the next backtracking trial)
        const double rb = sobolev(b);
        load_weights(cx.a);
        T *V = buf(B_V), *G = buf(B_G);
        const S pg = pass(true, bx, -1, -1, -1, B_Y, noprep, [=](int c, int gi, int gj, long long, int, T v, T yv) {
            const T e = v - yv;
            put(V, c, gi, gj, e);
            return e * e;
        });
        const S gval = reduce(pg, 2);
        if (!alive) return;
        const S pgg = pass(false, B_V, -1, -1, -1, -1, noprep, [=](int c, int gi, int gj, long long, int, T v, T) {
            const T gg = T(2) * v;
            put(G, c, gi, gj, gg);
            return gg * gg;
        });
        const S ggs = reduce(pgg, 3);
        if (!alive) return;
        passes += 2;
        loss = Sc::to_double(gval) + rb;
        gxn = sqrt(Sc::to_double(ggs));
        if (!isfinite(loss) || !isfinite(gxn)) {
            if (tid() == 0) raise(ST_NONFINITE);
            alive = false;
        }
    }

    // CG (Algorithm 1, step 2) on grad^2_x h(x, b) q = rhs with x in buffer bx,
    // rhs in brhs and q in B_Q (taken as zero when zero_start).  The direction
    // update p = r + beta p of iteration k is fused into the B p pass of
    // iteration k+1: each stage holds r and the previous p, combined in shared
    // memory, and the strip's own rows of p are written back.  Element-wise
    // updates run over whole padded buffers (ghosts stay current); sums count
    // image pixels only.  Returns iterations.
    __device__ int cg(const T *b, int bx, int brhs, double delta, int max_iters, bool zero_start, double &res,
                      int &capped, long long &passes)
    {
        if constexpr (kFFT) {
            if (cx.fr2c) return cg_r2c(b, bx, brhs, delta, max_iters, zero_start, res, capped, passes);
        }
        load_weights(b);
        T *R = buf(B_R), *HP = buf(B_HP), *Q = buf(B_Q);
        const T *RHS = buf(brhs);
        int pc = B_P0, po = B_P1;
        if (!zero_start) {
            hess_vec(bx, B_Q, B_HP, nullptr);
            if (!sync()) return 0;
            passes += gram() ? 1 : 2;
        }
        auto interior = [&](int row, int j) {
            const int pi = row % cx.Hp;
            return pi >= cx.Gy && pi < cx.Gy + cx.H && j >= cx.Gx && j < cx.Gx + cx.W;
        };
        S rrp = Sc::zero();
        {
            T *PCb = buf(pc);
            for (int row = gw(); row < cx.C * cx.Hp; row += TW()) {
                const long long rb = (long long)row * cx.Wp;
                T s = T(0);
                for (int j0 = 0; j0 < cx.Wp; j0 += 32 * EWB) {
                    T v[EWB];
#pragma unroll
                    for (int u = 0; u < EWB; ++u) {
                        const int j = j0 + u * 32 + lane;
                        v[u] = j < cx.Wp ? (zero_start ? __ldcg(RHS + rb + j) : __ldcg(RHS + rb + j) - __ldcg(HP + rb + j))
                                         : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < EWB; ++u) {
                        const int j = j0 + u * 32 + lane;
                        if (j < cx.Wp) {
                            if (zero_start) Q[rb + j] = T(0);
                            R[rb + j] = v[u];
                            PCb[rb + j] = v[u];
                            if (interior(row, j)) s += v[u] * v[u];
                        }
                    }
                }
                rrp = Sc::addv(rrp, s);
            }
        }
        S rr = reduce(rrp, 4);
        if (!alive) return 0;
        const S delta2 = Sc::from_double(delta * delta);
        int it = 0;
        capped = 0;
        bool first = true;
        T beta = T(0);
        T *U = buf(B_U);
        while (!Sc::le(rr, delta2) && it < max_iters) {
            // phase A: p (fused update unless first) and U = B p
            T *PW = buf(pc);
            const T bt = beta;
            const int BWl = cx.BW, r = cx.r, r4 = cx.r4;
            auto combine = [=](int st, int c, int row0, int col0) {
                const int n = NX * BWl;
                for (int e = lane; e < n; e += 32) sb0[e] = sb0[e] + bt * sb1()[e];
                __syncwarp();
                // the strip's own rows (tile rows r .. r+MR-1) that this stage owns
                const int gj = col0 + lane;
                for (int m = 0; m < MR; ++m) {
                    const int t = r + m;
                    if (t < st * PC || t >= (st + 1) * PC) continue;
                    const int gi = row0 + m;
                    if (gi < cx.H && gj < cx.W) put(PW, c, gi, gj, sb0[(t - st * PC) * BWl + r4 + lane]);
                }
            };
            auto epiU = [=](int c, int gi, int gj, long long, int, T v, T) { put(U, c, gi, gj, v); return T(0); };
            if (gram()) {              // p = r + beta p over the whole padded buffer (B p is not needed)
                if (!first) {
                    const T *Rr = buf(B_R), *Po = buf(po);
                    for (long long e = gstart(); e < cx.Np; e += gstride()) PW[e] = __ldcg(Rr + e) + bt * __ldcg(Po + e);
                }
            } else if (first) {
                pass(true, pc, -1, -1, -1, -1, noprep, epiU);
            } else {
                pass(true, B_R, po, -1, -1, -1, combine, epiU);
            }
            if (!sync()) return it;
            // phase B: HP = B^T U + alpha D^T(phi''(D x) . D p); <p, HP>
            const S php = reduce(hess_vec_b(bx, pc, B_HP, nullptr), 5);
            if (!alive) return it;
            passes += gram() ? 1 : 2;
            if (!Sc::finite(php)) {
                if (tid() == 0) raise(ST_NONFINITE);
                alive = false;
                return it;
            }
            if (!Sc::positive(php)) { capped = 1; break; }
            const T a = (T)Sc::to_elem(Sc::div(rr, php));
            S rn = Sc::zero();
            {
                const T *PCr = buf(pc);
                for (int row = gw(); row < cx.C * cx.Hp; row += TW()) {
                    const long long rb = (long long)row * cx.Wp;
                    T s = T(0);
                    for (int j0 = 0; j0 < cx.Wp; j0 += 32 * EWB) {
                        T pv[EWB], qv[EWB], rv[EWB], hv[EWB];
#pragma unroll
                        for (int u = 0; u < EWB; ++u) {
                            const int j = j0 + u * 32 + lane;
                            if (j < cx.Wp) {
                                pv[u] = __ldcg(PCr + rb + j);
                                qv[u] = __ldcg(Q + rb + j);
                                rv[u] = __ldcg(R + rb + j);
                                hv[u] = __ldcg(HP + rb + j);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < EWB; ++u) {
                            const int j = j0 + u * 32 + lane;
                            if (j < cx.Wp) {
                                Q[rb + j] = qv[u] + a * pv[u];
                                const T r2 = rv[u] - a * hv[u];
                                R[rb + j] = r2;
                                if (interior(row, j)) s += r2 * r2;
                            }
                        }
                    }
                    rn = Sc::addv(rn, s);
                }
            }
            const S rr_new = reduce(rn, 6);
            if (!alive) return it;
            ++it;
            if (!Sc::finite(rr_new)) {
                if (tid() == 0) raise(ST_NONFINITE);
                alive = false;
                return it;
            }
            if (Sc::le(rr_new, delta2)) { rr = rr_new; break; }
            beta = (T)Sc::to_elem(Sc::div(rr_new, rr));
            rr = rr_new;
            po = pc;
            pc = (pc == B_P0) ? B_P1 : B_P0;
            first = false;
        }
        res = sqrt(Sc::to_double(rr));
        if (!Sc::le(rr, delta2)) capped = 1;
        return it;
    }

    // CG of Algorithm 1 (step 2) on the real-to-complex pipeline: per
    // iteration the direction update with its forward row transforms, the
    // column phase, the inverse row transforms with the TV Hessian term and
    // <p, H p>, then the same element-wise update of q and r as cg()
    __device__ int cg_r2c(const T *b, int bx, int brhs, double delta, int max_iters, bool zero_start, double &res,
                      int &capped, long long &passes)
    {
        load_weights(b);
        T *R = buf(B_R), *HP = buf(B_HP), *Q = buf(B_Q);
        const T *RHS = buf(brhs);
        int pc = B_P0, po = B_P1;
        if (!zero_start) {             // HP = H q for the initial residual
            rows_r2c(RF_FWD, B_Q, -1, -1, -1, T(0));
            if (!sync()) return 0;
            cols_r2c();
            if (!sync()) return 0;
            rows_r2c(RF_HESS, B_Q, bx, B_HP, -1, T(0));
            if (!sync()) return 0;
            passes += 1;
        }
        auto interior = [&](int row, int j) {
            const int pi = row % cx.Hp;
            return pi >= cx.Gy && pi < cx.Gy + cx.H && j >= cx.Gx && j < cx.Gx + cx.W;
        };
        S rrp = Sc::zero();
        {
            T *PCb = buf(pc);
            for (int row = gw(); row < cx.C * cx.Hp; row += TW()) {
                const long long rb = (long long)row * cx.Wp;
                T s = T(0);
                for (int j0 = 0; j0 < cx.Wp; j0 += 32 * EWB) {
                    T v[EWB];
#pragma unroll
                    for (int u = 0; u < EWB; ++u) {
                        const int j = j0 + u * 32 + lane;
                        v[u] = j < cx.Wp ? (zero_start ? __ldcg(RHS + rb + j) : __ldcg(RHS + rb + j) - __ldcg(HP + rb + j))
                                         : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < EWB; ++u) {
                        const int j = j0 + u * 32 + lane;
                        if (j < cx.Wp) {
                            if (zero_start) Q[rb + j] = T(0);
                            R[rb + j] = v[u];
                            PCb[rb + j] = v[u];
                            if (interior(row, j)) s += v[u] * v[u];
                        }
                    }
                }
                rrp = Sc::addv(rrp, s);
            }
        }
        S rr = reduce(rrp, 4);
        if (!alive) return 0;
        const S delta2 = Sc::from_double(delta * delta);
        int it = 0;
        capped = 0;
        bool first = true;
        T beta = T(0);
        while (!Sc::le(rr, delta2) && it < max_iters) {
            // p = r + beta p (p = r, already in place, at the first iteration)
            // with its forward row transforms; the column phase; H p and <p, H p>
            if (first) rows_r2c(RF_FWD, pc, -1, -1, -1, T(0));
            else rows_r2c(RF_CGP, B_R, po, pc, -1, beta);
            if (!sync()) return it;
            cols_r2c();
            if (!sync()) return it;
            const S php = reduce(rows_r2c(RF_HESS, pc, bx, B_HP, -1, T(0)), 5);
            if (!alive) return it;
            passes += 1;
            if (!Sc::finite(php)) {
                if (tid() == 0) raise(ST_NONFINITE);
                alive = false;
                return it;
            }
            if (!Sc::positive(php)) { capped = 1; break; }
            const T a = (T)Sc::to_elem(Sc::div(rr, php));
            S rn = Sc::zero();
            {
                // 16-byte vectors: the padded pitch, the ghost width and W are
                // multiples of 4, so a vector is wholly interior or wholly ghost
                constexpr int V = 1;
                const float4 *P4 = reinterpret_cast<const float4 *>(buf(pc));
                const float4 *H4 = reinterpret_cast<const float4 *>(HP);
                float4 *Q4 = reinterpret_cast<float4 *>(Q), *R4 = reinterpret_cast<float4 *>(R);
                const int w4 = cx.Wp >> 2, g4 = cx.Gx >> 2, e4 = (cx.Gx + cx.W) >> 2;
                for (int row = gw(); row < cx.C * cx.Hp; row += TW()) {
                    const long long rb = (long long)row * w4;
                    const int pi = row % cx.Hp;
                    const bool irow = pi >= cx.Gy && pi < cx.Gy + cx.H;
                    T s = T(0);
                    for (int j0 = lane; j0 < w4; j0 += 32 * V) {
                        float4 pv[V], qv[V], rv[V], hv[V];
#pragma unroll
                        for (int u = 0; u < V; ++u) {
                            const int j = j0 + u * 32;
                            if (j < w4) {
                                pv[u] = __ldcg(P4 + rb + j);
                                qv[u] = __ldcg(Q4 + rb + j);
                                rv[u] = __ldcg(R4 + rb + j);
                                hv[u] = __ldcg(H4 + rb + j);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < V; ++u) {
                            const int j = j0 + u * 32;
                            if (j < w4) {
                                Q4[rb + j] = make_float4(qv[u].x + a * pv[u].x, qv[u].y + a * pv[u].y,
                                                         qv[u].z + a * pv[u].z, qv[u].w + a * pv[u].w);
                                const float4 r2 = make_float4(rv[u].x - a * hv[u].x, rv[u].y - a * hv[u].y,
                                                              rv[u].z - a * hv[u].z, rv[u].w - a * hv[u].w);
                                R4[rb + j] = r2;
                                if (irow && j >= g4 && j < e4)
                                    s += (r2.x * r2.x + r2.y * r2.y) + (r2.z * r2.z + r2.w * r2.w);
                            }
                        }
                    }
                    rn = Sc::addv(rn, s);
                }
            }
            const S rr_new = reduce(rn, 6);
            if (!alive) return it;
            ++it;
            if (!Sc::finite(rr_new)) {
                if (tid() == 0) raise(ST_NONFINITE);
                alive = false;
                return it;
            }
            if (Sc::le(rr_new, delta2)) { rr = rr_new; break; }
            beta = (T)Sc::to_elem(Sc::div(rr_new, rr));
            rr = rr_new;
            po = pc;
            pc = (pc == B_P0) ? B_P1 : B_P0;
            first = false;
        }
        res = sqrt(Sc::to_double(rr));
        if (!Sc::le(rr, delta2)) capped = 1;
        return it;
    }

    // out[c,p,q] = sum_ij x[c,i-p+r,j-q+r] (B v)[c,i,j] + v[c,i-p+r,j-q+r] (B x - y)[c,i,j]
    // (Algorithm 1, step 3, with the sign of Eq. 3.2: z = -out (+ grad r(b)));
    // x, v in buffers bx, bv; written to zout; returns ||zout||^2
    __device__ double cross(const T *b, int bx, int bv, T *zout, bool negate, bool add_r, long long &passes)
    {
        load_weights(b);
        T *U = buf(B_U), *V = buf(B_V);
        const int r = cx.r, K = cx.K, KK = K * K, H = cx.H, W = cx.W;
        const int CKK = cx.C * KK;
        S *zall = reinterpret_cast<S *>(cx.zpart);
        S *zp = zall + (long long)gw() * CKK;
        if constexpr (!kFFT) {         // per-warp lag-sum rows (the direct path's phase K2)
            for (int e = lane; e < CKK; e += 32) zp[e] = Sc::zero();
        }
        // phase K1: U = B v, V = B x - y (image pixels only: phase K2 reads
        // interiors).  The stages of v and then of x run through the same
        // double buffer.  On the FFT path: two passes.
        if (kFFT) {
            pass(true, bv, -1, -1, -1, -1, noprep, [=](int c, int gi, int gj, long long, int, T v, T) {
                U[pidx(c, gi, gj)] = v;
                return T(0);
            });
            pass(true, bx, -1, -1, -1, B_Y, noprep, [=](int c, int gi, int gj, long long, int, T v, T yv) {
                V[pidx(c, gi, gj)] = v - yv;
                return T(0);
            });
        } else if (!tmafail && alive) {
            if (lane == 0) fence_proxy_async();
            for (int s = gw(); s < cx.nstrips; s += TW()) {
                int c, row0, col0;
                strip_of(s, c, row0, col0);
                T au[MR], av[MR];
#pragma unroll
                for (int m = 0; m < MR; ++m) { au[m] = T(0); av[m] = T(0); }
                issue(0, bv, c, row0, col0, 0, bytes_i(), [&](uint64_t *mb) { box_i(tF(), B_Y, c, row0, col0, mb); });
                bool ok = true;
                for (int k = 0; k < 2 * ns(); ++k) {
                    if (!land(k & 1)) { ok = false; break; }
                    if (k + 1 < 2 * ns()) {
                        const int kn = k + 1;
                        issue(kn, kn < ns() ? bv : bx, c, row0, col0, (kn < ns() ? kn : kn - ns()) * PC, 0u,
                              [](uint64_t *) {});
                    }
                    if (k < ns()) corr_on(sb(k & 1), true, c, k * PC, au);
                    else corr_on(sb(k & 1), true, c, (k - ns()) * PC, av);
                    fence_proxy_async_smem();
                    __syncwarp();
                }
                if (!ok) break;
                const int gj = col0 + lane;
#pragma unroll
                for (int m = 0; m < MR; ++m) {
                    const int gi = row0 + m;
                    if (gi < H && gj < W) {
                        const long long o = pidx(c, gi, gj);
                        U[o] = au[m];
                        V[o] = av[m] - tF()[m * 32 + lane];
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
            }
        }
        if (!sync()) return 0.0;
        if (gram()) {   // FFT path: all lags from one spectrum product, then sign and Sobolev term
            if (!fft_cross(bx, bv)) return 0.0;
            for (long long e = gstart(); e < CKK; e += gstride()) {
                const int c = (int)(e / KK), pq = (int)(e - (long long)c * KK), p = pq / K, q = pq - p * K;
                const int i = ((p - r) % H + H) % H, j = ((q - r) % W + W) % W;
                double zz = (double)__ldcg(cx.fout + (long long)c * cx.HW + (long long)i * W + j) + cross_off()[c];
                if (negate) zz = -zz;
                if (add_r) zz += grad_sobolev_elem(b, (int)e);
                zout[e] = (T)zz;
            }
            passes += 4;
        } else {
        // phase K2: lag sums of this warp's strips, by stages of PC lag rows.
        // Lag p and strip row m read tile row m + 2r - p, so the stage of lags
        // p0 .. p0+PC-1 holds tile rows from 2r - p0 - PC + 1 (NX rows) of x
        // (sb0) and v (sb1()).  A lane owns one lag row p and QB consecutive lag
        // columns q0..q0+QB-1; along each strip row the x and v windows slide
        // through registers (one new shared load each per column).
        const int nqb = (K + QB - 1) / QB;
        if (!tmafail) {
            if (lane == 0) fence_proxy_async();
            for (int s = gw(); s < cx.nstrips; s += TW()) {
                int c, row0, col0;
                strip_of(s, c, row0, col0);
                bool ok = true;
                for (int st = 0; st < ns(); ++st) {
                    const int p0 = st * PC, t0 = 2 * r - p0 - PC + 1;
                    if (lane == 0) {
                        uint64_t *mb = &mbar()[0];
                        mbar_expect_tx(mb, 2 * bytes_s() + (st == 0 ? 2 * bytes_i() : 0u));
                        box_s(sb0, bx, c, row0, col0, t0, mb);
                        box_s(sb1(), bv, c, row0, col0, t0, mb);
                        if (st == 0) {
                            box_i(t1(), B_U, c, row0, col0, mb);
                            box_i(t2(), B_V, c, row0, col0, mb);
                        }
                    }
                    if (!land(0)) { ok = false; break; }
                    if (st == 0) {
                        // pixels outside the image (ragged strips) must not contribute
                        const int gj = col0 + lane;
                        for (int m = 0; m < MR; ++m) {
                            if (row0 + m >= H || gj >= W) {
                                t1()[m * 32 + lane] = T(0);
                                t2()[m * 32 + lane] = T(0);
                            }
                        }
                        __syncwarp();
                    }
                    const int np = K - p0 < PC ? K - p0 : PC;
                    const int units = np * nqb;
                    for (int u = lane; u < units; u += 32) {
                        const int p = p0 + u / nqb, q0 = (u % nqb) * QB;
                        S acc[QB];
#pragma unroll
                        for (int k = 0; k < QB; ++k) acc[k] = Sc::zero();
                        for (int m = 0; m < MR; ++m) {
                            const int srow = m + p0 + PC - 1 - p;     // = tile row m + 2r - p, minus t0
                            const T *rx = sb0 + srow * cx.BW + off();
                            const T *rv = sb1() + srow * cx.BW + off();
                            const T *ur = t1() + m * 32, *vr = t2() + m * 32;
                            const int c0 = 2 * r - q0;       // column of lag q0 at j = 0
                            T wx[QB], wv[QB], af[QB];
#pragma unroll
                            for (int k = 0; k < QB; ++k) af[k] = T(0);
#pragma unroll
                            for (int k = 1; k < QB; ++k) {
                                const int col = c0 - k >= 0 ? c0 - k : 0;   // only unused lags clamp
                                wx[(QB - k) % QB] = rx[col];
                                wv[(QB - k) % QB] = rv[col];
                            }
                            for (int j0 = 0; j0 < 32; j0 += QB) {
#pragma unroll
                                for (int jj = 0; jj < QB; ++jj) {
                                    const int j = j0 + jj;
                                    wx[jj] = rx[c0 + j];
                                    wv[jj] = rv[c0 + j];
                                    const T uu = ur[j], vv = vr[j];
#pragma unroll
                                    for (int k = 0; k < QB; ++k)
                                        af[k] = fma(wx[(jj - k + QB) % QB], uu, fma(wv[(jj - k + QB) % QB], vv, af[k]));
                                }
                            }
#pragma unroll
                            for (int k = 0; k < QB; ++k) acc[k] = Sc::addv(acc[k], af[k]);
                        }
#pragma unroll
                        for (int k = 0; k < QB; ++k)
                            if (q0 + k < K) zp[c * KK + p * K + q0 + k] = Sc::add(zp[c * KK + p * K + q0 + k], acc[k]);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                }
                if (!ok) break;
            }
        }
        if (!sync()) return 0.0;
        // phase K3: one warp per kernel entry sums the per-warp rows in a fixed
        // order (lane l takes rows l, l+32, ...; then the shuffle tree), then
        // applies the sign and the Sobolev term
        for (int e = gw(); e < CKK; e += TW()) {
            S s = Sc::zero();
#pragma unroll 4
            for (int w = lane; w < TW(); w += 32) s = Sc::add(s, Sc::load_cg(zall + (long long)w * CKK + e));
            s = warp_sum<T>(s);
            if (lane == 0) {
                double zz = Sc::to_double(s);
                if (negate) zz = -zz;
                if (add_r) zz += grad_sobolev_elem(b, e);
                zout[e] = (T)zz;
            }
        }
        passes += 4;   // B v, B x and the two lag correlations
        }
        if (!sync()) return 0.0;
        S s = Sc::zero();
        for (int e = tid(); e < CKK; e += blockDim.x) {
            const T zv = __ldcg(zout + e);
            s = Sc::addv(s, zv * zv);
        }
        return Sc::to_double(block_sum<T>(s, red()));
    }

    // ------------------------------------------------------------ MAID
    // Upper iterations of Algorithm 2: one (jb.max_steps <= 1) or a whole run
    // of up to jb.max_steps in this launch, stopping at the stop rule or when
    // a step exhausts its backtracking rounds.  Every CTA runs the same control
    // flow on identical reduction results.  x~(b_k) lives in B_XK between the
    // steps; the trial solutions go to B_XT.  Register economy: the run's
    // constant parameters are read from the job (or its device-resident home)
    // where used, the report is accumulated in shared memory by thread 0, and
    // only the adaptive quantities and the current comparison terms stay in
    // registers.
    __device__ void maid(const Job<T> &jb)
    {
        const MaidIn &M = jb.maid_home ? *jb.maid_home : jb.maid;   // constant fields
        MaidRep &R = g_rep;
        double eps = M.eps, delta = M.delta, step = M.step;
        int k = M.k;
        T *b = jb.bio;
        const int CKK = cx.C * cx.K * cx.K;
        const int steps = jb.max_steps > 1 ? jb.max_steps : 1;
        long long passes = 0;
        bool stopped = (M.eps_stop > 0.0 && eps <= M.eps_stop) || M.halted;   // stop rule of Sec. 4.2
        bool halted = false, any_accepted = false, accepted = false;
        int rounds = 0, ran = 0, n_accepted = 0;
        if (tid() == 0) R = MaidRep{};
        __syncthreads();
        if (!stopped) {
            import_dense(jb.x, B_XK);
            if (!sync()) stopped = true;
        }
        for (int sidx = 0; sidx < steps && alive && !stopped && !halted; ++sidx) {
            accepted = false;
            rounds = 0;
            // a step that exhausts its rounds leaves x~ as it was (the solves
            // refine B_XK in place): keep a copy when a later step can fail
            if (steps > 1) copy_buf(B_IN1, -1, B_XK);
            if (tid() == 0) { R.ll_iters = R.cg_iters = R.ll_capped = R.cg_capped = R.trials = 0; }
            int j = M.max_bt;
            for (int round = 0; round < M.max_rounds && alive && !stopped; ++round, ++j) {
                rounds = round + 1;
                // InexactGradient(b_k, eps_k, delta_k)
                double gn = 0.0, res = 0.0;
                int it = lower_solve(b, B_XK, B_XK, eps, M.ll_max_iters, gn, passes);
                if (tid() == 0) { R.ll_iters += it; R.fused += it; if (gn > eps) R.ll_capped = 1; }
                if (!sync()) break;
                double l0 = 0.0, gx0 = 0.0;
                upper_loss(b, B_XK, l0, gx0, passes);
                if (!alive) break;
                int capped = 0;
                it = cg(b, B_XK, B_G, delta, M.cg_max_iters, true, res, capped, passes);
                if (tid() == 0) { R.cg_iters += it; R.fused += it; if (capped) R.cg_capped = 1; }
                if (!alive) break;
                if (!sync()) break;
                const double zz = cross(b, B_XK, B_Q, cx.ZK, true, true, passes);
                if (!alive) break;
                if (tid() == 0) R.znorm = sqrt(zz);
                if (!isfinite(zz)) {
                    if (tid() == 0) raise(ST_NONFINITE);
                    alive = false;
                    break;
                }
                bool done = false;
                for (int i = 0; i < j; ++i) {
                    if (tid() == 0) ++R.trials;
                    // b' = b - step z
                    for (long long e = gstart(); e < CKK; e += gstride())
                        cx.BT[e] = (T)((double)__ldcg(b + e) - step * (double)__ldcg(cx.ZK + e));
                    if (!sync()) break;
                    double g1 = 0.0;
                    it = lower_solve(cx.BT, B_XK, B_XT, eps, M.ll_max_iters, g1, passes);
                    if (tid() == 0) { R.ll_iters += it; R.fused += it; if (g1 > eps) R.ll_capped = 1; }
                    if (!sync()) break;
                    double l1 = 0.0, gx1 = 0.0;
                    upper_loss(cx.BT, B_XT, l1, gx1, passes);
                    if (!alive) break;
                    // psi of Eq. 3.4 with eps_bar = eps_k
                    const double eb = eps;
                    const double psi = l1 + gx1 * eb + 0.5 * M.L_gx * eb * eb - l0 + gx0 * eb + M.lambda * step * zz;
                    if (tid() == 0) R.psi = psi;
                    if (psi <= 0.0) {
                        for (long long e = gstart(); e < CKK; e += gstride()) b[e] = __ldcg(cx.BT + e);
                        copy_buf(B_XK, -1, B_XT);
                        if (tid() == 0) { R.loss = l1; R.gxn = gx1; }
                        eps *= M.nu_up;
                        delta *= M.nu_up;
                        step *= M.rho_up;
                        k += 1;
                        accepted = true;
                        done = true;
                        break;
                    }
                    step *= M.rho_down;
                }
                if (done || !alive) break;
                if (tid() == 0) { R.loss = l0; R.gxn = gx0; }
                eps *= M.nu_down;
                delta *= M.nu_down;
                if (M.eps_stop > 0.0 && eps <= M.eps_stop) stopped = true;
            }
            if (!alive) break;
            ++ran;
            if (accepted) {
                any_accepted = true;
                ++n_accepted;
                // the next step reads b_{k+1}, written above by other CTAs
                if (sidx + 1 < steps && !sync()) break;
            } else if (!stopped) {
                halted = true;         // a step exhausted its rounds: the run ends here
            }
        }
        // x~ and q back to the caller (x unchanged unless a step was accepted)
        if (alive && ran > 0 && sync()) {
            if (any_accepted) export_dense(halted ? B_IN1 : B_XK, (T *)jb.x);
            export_dense(B_Q, jb.q);
        }
        __syncthreads();               // thread 0's report entries are complete
        if (tid() == 0 && bid == 0) {
            if (jb.maid_home) {        // device-resident state for a later launch (same bytes when unchanged)
                MaidIn *h = jb.maid_home;
                h->eps = eps; h->delta = delta; h->step = step; h->k = k;
                if (halted && alive) h->halted = 1;
            }
            if (cx.totals && ran > 0) {
                MaidTotals *t = cx.totals;
                t->fused_iters += R.fused;
                t->conv_passes += passes;
                t->upper_iters += ran;
                t->accepted += n_accepted;
            }
            DevOut *o = cx.out;
            o->accepted = accepted; o->rounds = rounds; o->trials = R.trials;
            o->ll_iters = R.ll_iters; o->cg_iters = R.cg_iters; o->ll_capped = R.ll_capped; o->cg_capped = R.cg_capped;
            o->k = k; o->eps = eps; o->delta = delta; o->step = step;
            o->loss = R.loss; o->gradx_norm = R.gxn; o->znorm = R.znorm; o->psi = R.psi;
            o->conv_passes = passes; o->stopped = stopped;
            o->iters = ran;
        }
    }
};

// The program of one call (selected by jb.mode) on one problem; every CTA of
// the problem's grid or group runs it.
template <typename T, bool FFTP>
__device__ __forceinline__ void run_program(Eng<T, FFTP> &e, const Ctx<T> &cx, const Job<T> &jb)
{
    const bool lead = threadIdx.x == 0 && e.bid == 0;
    long long passes = 0;
    switch (jb.mode) {
    case M_IMPORT_Y: e.import_dense(jb.x, B_Y); break;
    case M_APPLY_B:
    case M_APPLY_BT:
        e.import_dense(jb.x, B_IN1);
        e.load_weights(jb.b);
        if (e.sync()) e.apply(B_IN1, jb.xo, jb.mode == M_APPLY_BT);
        break;
    case M_GRAD_LOWER:
        e.import_dense(jb.x, B_XK);
        if (e.sync()) e.grad_lower(jb.b, B_XK, jb.xo);
        break;
    case M_HESS_VEC:
        e.import_dense(jb.x, B_XK);
        e.import_dense(jb.v, B_IN1);
        e.load_weights(jb.b);
        if (e.sync()) e.hess_vec(B_XK, B_IN1, B_HP, jb.xo);
        break;
    case M_LOWER_SOLVE: {
        if (jb.y) e.import_dense(jb.y, B_Y);
        e.import_dense(jb.x, B_XK);
        double gn = 0.0;
        int it = 0;
        if (e.sync()) {
            it = e.lower_solve(jb.b, B_XK, B_XK, jb.eps, jb.max_iters, gn, passes);
            if (e.sync()) e.export_dense(B_XK, jb.xo);
        }
        if (lead) {
            cx.out->iters = it; cx.out->gradnorm = gn; cx.out->capped = gn > jb.eps;
            cx.out->conv_passes = passes;
        }
        break;
    }
    case M_UPPER_LOSS: {
        e.import_dense(jb.x, B_XK);
        double loss = 0.0, gxn = 0.0;
        if (e.sync()) {
            e.upper_loss(jb.b, B_XK, loss, gxn, passes);
            if (e.alive && jb.xo) e.export_dense(B_G, jb.xo);
        }
        if (lead) { cx.out->loss = loss; cx.out->gradx_norm = gxn; cx.out->conv_passes = passes; }
        break;
    }
    case M_HYPERGRAD: {
        const bool given = jb.v != nullptr;
        e.import_dense(jb.x, B_XK);
        e.import_dense(jb.q, B_Q);
        if (given) e.import_dense(jb.v, B_IN1);
        if (!e.sync()) break;
        double gxn = 0.0, loss = 0.0;
        int rhs = B_IN1;
        if (!given) {
            e.upper_loss(jb.b, B_XK, loss, gxn, passes);
            if (!e.alive) break;
            rhs = B_G;
        }
        double res = 0.0;
        int capped = 0;
        const int it = e.cg(jb.b, B_XK, rhs, jb.delta, jb.max_iters, false, res, capped, passes);
        if (!e.alive) break;
        if (!e.sync()) break;
        const double zz = e.cross(jb.b, B_XK, B_Q, jb.z, true, !given, passes);
        if (e.alive) e.export_dense(B_Q, jb.q);
        if (lead) {
            cx.out->cg_iters = it; cx.out->resnorm = res; cx.out->capped = capped;
            cx.out->znorm = sqrt(zz); cx.out->conv_passes = passes;
        }
        break;
    }
    case M_CROSS:
        e.import_dense(jb.x, B_XK);
        e.import_dense(jb.v, B_IN1);
        if (e.sync()) e.cross(jb.b, B_XK, B_IN1, jb.z, false, false, passes);
        break;
    case M_MAID: e.maid(jb); break;
    case M_WAIT_SELFTEST:
        // diagnostic: CTA 0 never arrives, so every other CTA's bounded wait at
        // this barrier runs out and records ST_TIMEOUT
        if (e.bid != 0) e.sync();
        break;
    default: break;
    }
    e.drain();
    if (threadIdx.x == 0 && e.bid == 0) cx.out->barriers = (int)e.epoch;
}

// Dynamic shared memory: the TMA destinations need 128-byte alignment, which
// the kernel checks (a launch that does not get it reports ST_TIMEOUT-free
// failure through the status word and returns).
#define ADP_KERNEL_SMEM extern __shared__ __align__(128) unsigned char smem_raw[]

// One problem per launch: the launch record lives in parameter space.
template <typename T, bool FFTP = false>
__global__ void __launch_bounds__((FFTP ? FFT_WARPS : MAXNW) * 32, FFTP ? FFT_CTAS_PER_SM : 1)
    adp_kernel(const __grid_constant__ Ctx<T> cx,
                                                            const __grid_constant__ Job<T> jb)
{
    ADP_KERNEL_SMEM;
    if ((reinterpret_cast<uintptr_t>(smem_raw) & 127) != 0) {
        if (threadIdx.x == 0) atomicCAS(&cx.out->status, ST_OK, ST_ALIGN);
        return;
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) cx.out->t_start = (long long)globaltimer_ns();
    Eng<T, FFTP> e(cx, &cx, gridDim.x, blockIdx.x, smem_raw);
    run_program<T, FFTP>(e, cx, jb);
    if (threadIdx.x == 0 && blockIdx.x == 0) cx.out->t_end = (long long)globaltimer_ns();
}

// Many problems per launch: CTAs first[g] .. first[g+1]-1 form problem g's
// group (its own barrier counter, reductions and result record); the launch
// records live in global memory (tensor maps included, 64-byte aligned).
template <typename T>
__global__ void __launch_bounds__(MAXNW * 32, 1) adp_kernel_batched(const Ctx<T> *__restrict__ ctxs,
                                                                    const Job<T> *__restrict__ jobs,
                                                                    const int *__restrict__ first, int n)
{
    ADP_KERNEL_SMEM;
    int g = 0;
    while (g + 1 < n && (int)blockIdx.x >= __ldg(first + g + 1)) ++g;
    const int f0 = __ldg(first + g), nb = __ldg(first + g + 1) - f0;
    // the record in shared memory (its fields are read all over the engine);
    // the tensor maps are used from global memory, where TMA can read them
    __shared__ __align__(64) unsigned char ctx_sh[sizeof(Ctx<T>)];
    for (int i = threadIdx.x; i < (int)(sizeof(Ctx<T>) / 4); i += blockDim.x)
        reinterpret_cast<int *>(ctx_sh)[i] = __ldg(reinterpret_cast<const int *>(ctxs + g) + i);
    __syncthreads();
    const Ctx<T> &cx = *reinterpret_cast<const Ctx<T> *>(ctx_sh);
    if ((reinterpret_cast<uintptr_t>(smem_raw) & 127) != 0) {
        if (threadIdx.x == 0) atomicCAS(&cx.out->status, ST_OK, ST_ALIGN);
        return;
    }
    if (threadIdx.x == 0 && blockIdx.x == (unsigned)f0) cx.out->t_start = (long long)globaltimer_ns();
    Eng<T, false> e(cx, ctxs + g, nb, (int)blockIdx.x - f0, smem_raw);
    run_program<T, false>(e, cx, jobs[g]);
    if (threadIdx.x == 0 && blockIdx.x == (unsigned)f0) cx.out->t_end = (long long)globaltimer_ns();
}

} // namespace adp
