// Device building blocks of libadp: strip geometry, asynchronous halo loaders,
// the register-blocked direct correlation, deterministic FP64 reductions and
// the bounded grid barrier, plus the launch records (Ctx, Job) shared with the
// host code in adp.cu.
#pragma once

#include <cuda.h>          // CUtensorMap (type only; encoded on the host through the runtime's entry point)
#include <cuda_runtime.h>
#include <stdint.h>

namespace adp {

constexpr int MAXNW = 8;           // most warps per CTA (direct correlation)
constexpr int MAXNW_FFT = 16;      // warps per CTA the static arrays allow
constexpr int FFT_WARPS = 16;      // warps per CTA of the FFT-path kernel
constexpr int FFT_CTAS_PER_SM = 1; // its CTAs per SM
constexpr int MAXC = 64;           // channels supported (per-channel step cache)
constexpr int KMAX = 63;           // largest odd kernel size supported
constexpr int NSLOT = 8;           // scalar reduction slots
constexpr int SMEM_STATIC_MARGIN = 8 * 1024;   // static shared memory of the kernels is below this
constexpr int QB = 8;              // lag columns per lane in the kernel-gradient correlation

// Output rows per thread (a warp owns a strip of 32 columns x MR rows) and
// kernel rows per correlation chunk.
template <typename T> struct Cfg;
template <> struct Cfg<float>  { static constexpr int MR = 8, PC = 16; };
template <> struct Cfg<double> { static constexpr int MR = 4, PC = 8; };

// Status words shared with the host (values equal adp_status).
enum : int { ST_OK = 0, ST_NONFINITE = 4, ST_NOCONV = 5, ST_LSFAIL = 6, ST_TIMEOUT = 7, ST_ALIGN = 100 };

// Written by the device, copied to pinned host memory after each launch.
struct DevOut {
    int status;
    int iters, cg_iters, capped;
    double gradnorm, resnorm, loss, gradx_norm, znorm, psi;
    // MAID report and updated state
    int accepted, rounds, trials, ll_iters, ll_capped, cg_capped, k, pad;
    double eps, delta, step;
    long long conv_passes;       // number of full-image convolution passes executed
    int barriers, stopped;       // grid barriers executed by CTA 0; MAID stop rule fired
    long long t_start, t_end;    // global timer (ns) at the program's start and end in CTA 0
};

__host__ __device__ constexpr int round_up(int a, int m) { return (a + m - 1) / m * m; }

__device__ __forceinline__ int wrapi(int i, int n)
{
    int m = i % n;
    return m < 0 ? m + n : m;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *(const volatile int *)p;
}

// Grid-wide barrier for a cooperative launch.  Thread 0 of each CTA adds one
// to a monotonic arrival counter with release semantics and spins (acquire)
// until the counter reaches epoch * nblk (the CTAs sharing the counter: the
// whole grid, or one problem's group in a batched launch); the CTA's other threads are
// ordered by bar.sync on both sides.  The host zeroes the counter before each
// launch.  Every spin is bounded: after timeout_ns, or as soon as a CTA has
// raised a status, the waiter records ST_TIMEOUT (unless something else was
// recorded) and returns false, and the caller unwinds.
__device__ __forceinline__ bool grid_sync(unsigned *count, unsigned epoch, unsigned nblk, int *status,
                                          long long timeout_ns, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = epoch * nblk;
        red_release_add_u32(count, 1u);
        const uint64_t t0 = globaltimer_ns();
        unsigned spins = 0;
        while (ld_acquire_u32(count) < target) {
            if ((++spins & 255u) == 0u) {
                if (ld_volatile_i32(status) != ST_OK) { ok = 0; break; }
                if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
                    atomicCAS(status, ST_OK, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok && ld_volatile_i32(status) != ST_OK) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// ------------------------------------------------------------ scalars
// Reductions and the iteration control of the FP32 path run in float-float
// ("double-single") arithmetic: a value is an unevaluated sum hi + lo of two
// floats, updated with the error-free transformations TwoSum and TwoProd
// (Knuth; Dekker), which carry about 48 significant bits.  This keeps sums and
// dot products near FP64 accuracy while using only the FP32 pipes: on GB300 an
// FP64 instruction occupies the FP64 pipe for tens of cycles per warp.  The
// FP64 path (T = double) uses plain doubles.  Every reduction runs in a fixed
// order, so results are deterministic and identical in all CTAs.
struct __align__(8) ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// Quotient and square root: a fast first approximation, then one correction
// from the exact residual (computed with TwoProd), which restores float-float
// accuracy whatever the few-ulp error of the first step.
__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float q1 = __fdividef(a.hi, b.hi);
    const ff r = ff_add(a, ff_neg(ff_mul(b, ff{q1, 0.0f})));
    const float q2 = __fdividef(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ ff ff_sqrt(ff a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float s = __fmul_rn(a.hi, rsqrtf(a.hi));
    const ff r = ff_add(a, ff_neg(ff_mul(ff{s, 0.0f}, ff{s, 0.0f})));
    return fast_two_sum(s, __fdividef(r.hi, __fmul_rn(2.0f, s)));
}

// Arithmetic of reduction and control scalars for element type T.
template <typename T> struct Scal;
template <> struct Scal<float> {
    using S = ff;
    static __device__ __forceinline__ S zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ S of(float v) { return {v, 0.0f}; }
    static __device__ __forceinline__ S add(S a, S b) { return ff_add(a, b); }
    static __device__ __forceinline__ S addv(S a, float v) { return ff_add_f(a, v); }
    static __device__ __forceinline__ S mul(S a, S b) { return ff_mul(a, b); }
    static __device__ __forceinline__ S div(S a, S b) { return ff_div(a, b); }
    static __device__ __forceinline__ S sqroot(S a) { return ff_sqrt(a); }
    static __device__ __forceinline__ S shfl_down(S a, int o)
    {
        return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
    }
    static __device__ __forceinline__ float to_elem(S a) { return a.hi; }   // hi is hi + lo rounded
    static __device__ __forceinline__ double to_double(S a) { return (double)a.hi + (double)a.lo; }
    static __device__ __forceinline__ S from_double(double d)
    {
        const float hi = (float)d;
        return {hi, (float)(d - (double)hi)};
    }
    static __device__ __forceinline__ bool le(S a, S b)
    {
        const S d = ff_add(a, ff_neg(b));
        return d.hi < 0.0f || (d.hi == 0.0f && d.lo <= 0.0f);
    }
    static __device__ __forceinline__ bool positive(S a) { return a.hi > 0.0f; }
    static __device__ __forceinline__ bool finite(S a) { return isfinite(a.hi) && isfinite(a.lo); }
    static __device__ __forceinline__ S load_cg(const S *p)
    {
        const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
        return {v.x, v.y};
    }
};
template <> struct Scal<double> {
    using S = double;
    static __device__ __forceinline__ S zero() { return 0.0; }
    static __device__ __forceinline__ S of(double v) { return v; }
    static __device__ __forceinline__ S add(S a, S b) { return a + b; }
    static __device__ __forceinline__ S addv(S a, double v) { return a + v; }
    static __device__ __forceinline__ S mul(S a, S b) { return a * b; }
    static __device__ __forceinline__ S div(S a, S b) { return a / b; }
    static __device__ __forceinline__ S sqroot(S a) { return a > 0.0 ? sqrt(a) : 0.0; }
    static __device__ __forceinline__ S shfl_down(S a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
    static __device__ __forceinline__ double to_elem(S a) { return a; }
    static __device__ __forceinline__ double to_double(S a) { return a; }
    static __device__ __forceinline__ S from_double(double d) { return d; }
    static __device__ __forceinline__ bool le(S a, S b) { return a <= b; }
    static __device__ __forceinline__ bool positive(S a) { return a > 0.0; }
    static __device__ __forceinline__ bool finite(S a) { return isfinite(a); }
    static __device__ __forceinline__ S load_cg(const S *p) { return __ldcg(p); }
};

// Sum over a warp; lane 0 holds the result (fixed tree order).
template <typename T>
__device__ __forceinline__ typename Scal<T>::S warp_sum(typename Scal<T>::S v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Scal<T>::add(v, Scal<T>::shfl_down(v, o));
    return v;
}

// Deterministic CTA sum; every thread returns the same value.  `red` is a
// shared array of MAXNW scalars.
template <typename T>
__device__ __forceinline__ typename Scal<T>::S block_sum(typename Scal<T>::S v, typename Scal<T>::S *red)
{
    v = warp_sum<T>(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    typename Scal<T>::S t = Scal<T>::zero();
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) t = Scal<T>::add(t, red[w]);
    return t;
}

// FP64 CTA sum (small control quantities: kernel norms, the Sobolev term).
__device__ __forceinline__ double block_sum_d(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

// Grid totals.  Every CTA sums part[0..n) in the same fixed order (lane l of
// warp 0 takes entries l, l+32, ... and the lanes are combined by the shuffle
// tree), so all CTAs obtain identical bits.  The values come from other CTAs;
// warp 0 stages them into shared memory with asynchronous copies (one round
// trip through L2) in grid_issue, and grid_finish waits and sums, so callers
// can overlap the copies with other work without holding registers.
constexpr int GT_MAX = 512;          // largest grid the staging buffer holds

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// wait until at most n of this thread's most recent cp.async groups are pending
template <int n>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory"); }

// warp 0 only; entries are 8-byte scalars
template <typename T>
__device__ __forceinline__ void grid_issue(const typename Scal<T>::S *part, int n, typename Scal<T>::S *sbuf)
{
    for (int i = threadIdx.x & 31; i < n; i += 32) cp_async8(sbuf + i, part + i);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// warp 0 only; lane 0 returns the total
template <typename T>
__device__ __forceinline__ typename Scal<T>::S grid_finish(int n, const typename Scal<T>::S *sbuf)
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    typename Scal<T>::S s = Scal<T>::zero();
    for (int i = threadIdx.x & 31; i < n; i += 32) s = Scal<T>::add(s, sbuf[i]);
    return warp_sum<T>(s);
}

template <typename T>
__device__ __forceinline__ typename Scal<T>::S grid_total(const typename Scal<T>::S *part, int n,
                                                          typename Scal<T>::S *sbuf, typename Scal<T>::S *bcast)
{
    __syncthreads();
    if (threadIdx.x < 32) {
        grid_issue<T>(part, n, sbuf);
        const typename Scal<T>::S s = grid_finish<T>(n, sbuf);
        if (threadIdx.x == 0) *bcast = s;
    }
    __syncthreads();
    return *bcast;
}

// ------------------------------------------------------------ TMA
// Tiled bulk tensor copies (cp.async.bulk.tensor) into shared memory, with
// completion counted in bytes on a per-warp mbarrier.  The workspace is one
// 4D tensor [buffer][channel][padded row][padded column]; every tile the
// engine needs is a box of it.  The innermost coordinate is always a multiple
// of 4 elements (16 bytes).  Waits are bounded: after timeout_ns the waiter
// reports failure and the caller unwinds.

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// makes the initialised barriers visible to the async proxy (TMA completions)
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(mbar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait for the given phase parity of mbar; false when the budget ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, unsigned parity, long long timeout_ns)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) return false;
    }
}

// plain arrival (count 1) on an mbarrier, release semantics at CTA scope
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Untiled bulk copies (both addresses 16-byte aligned, bytes a multiple of
// 16): global to this CTA's shared memory, completion counted on mbar; and
// shared to global in a bulk group of the issuing thread.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
// tiled 2-D copies of a box of a 2-D tensor map (x innermost, 16-byte aligned)
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
                 "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the issuing thread's bulk groups: all have finished reading their shared sources
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and have completed their writes
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::
            "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(mbar))
        : "memory");
}

// Proxy fences.  Global: orders generic-proxy writes before later async-proxy
// (TMA) reads of them; taken by every writer before a grid barrier and by the
// issuing lane after it.  Shared: orders a lane's generic reads and writes of a
// staging buffer before the TMA that refills it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Register-blocked direct correlation of one 32-column x MR-row strip over
// one stage: PC consecutive kernel rows p0 .. p0+PC-1, kernel columns q0 .. K-1.
//   acc[m] += sum_{q0<=q<K} sum_{p<PC} w[q*Kp + p] * s[(m + p)*pitch + lj + q]
// s holds the PC + MR - 1 tile rows of the stage; w points at row p0 of a
// kernel stored column-major (w[q][p], p contiguous, rows zero-padded to Kp).
// Per kernel column the thread needs PC + MR - 1 values of its tile column and
// PC weights (vector loads, the same address in every lane); they are loaded
// one column ahead of the MR x PC FMAs that use them, so load latency
// overlaps arithmetic.  The weights are in shared memory, or in global memory
// read through L1 (coherent after the grid barrier that follows their
// writing); the caller's pointer provenance decides which loads are emitted.
template <typename T> struct Vec4;
template <> struct Vec4<float> { using V = float4; static constexpr int L = 4; };
template <> struct Vec4<double> { using V = double2; static constexpr int L = 2; };

template <typename T, int PC>
__device__ __forceinline__ void load_wchunk(const T *wq, T (&wv)[PC])
{
    using V = typename Vec4<T>::V;
    constexpr int L = Vec4<T>::L;
    const V *p = reinterpret_cast<const V *>(wq);
#pragma unroll
    for (int i = 0; i < PC / L; ++i) {
        const V v = p[i];
        if constexpr (L == 4) { wv[4 * i] = v.x; wv[4 * i + 1] = v.y; wv[4 * i + 2] = v.z; wv[4 * i + 3] = v.w; }
        else { wv[2 * i] = v.x; wv[2 * i + 1] = v.y; }
    }
}

template <typename T, int MR, int PC>
__device__ __forceinline__ void corr_stage(const T *__restrict__ s, int pitch, const T *w, int q0, int K,
                                           int Kp, int lj, T (&acc)[MR])
{
    constexpr int NX = PC + MR - 1;
    T xa[NX], wa[PC], xb[NX], wb[PC];
    int q = 0;
    auto load = [&](T (&xv)[NX], T (&wv)[PC]) {
        const T *col = s + lj + q;
#pragma unroll
        for (int i = 0; i < NX; ++i) xv[i] = col[i * pitch];
        load_wchunk<T, PC>(w + q * Kp, wv);
        ++q;
    };
    auto comp = [&](const T (&xv)[NX], const T (&wv)[PC]) {
#pragma unroll
        for (int p = 0; p < PC; ++p)
#pragma unroll
            for (int m = 0; m < MR; ++m) acc[m] = fma(wv[p], xv[m + p], acc[m]);
    };
    q = q0;
    if (q0 >= K) return;
    load(xa, wa);
    int qi = q0;
    for (; qi + 2 <= K; qi += 2) {
        load(xb, wb);
        comp(xa, wa);
        if (qi + 2 < K) load(xa, wa);
        comp(xb, wb);
    }
    if (qi < K) comp(xa, wa);
}

// phi' and phi'' of the regularisers (reg: 0 Huber, 1 sqrt, 2 quadratic);
// ig = 1/gamma for the Huber branch.  The FP32 path uses the reciprocal and the
// hardware reciprocal square root (a few ulp) instead of IEEE division.
__device__ __forceinline__ float rsqrt_t(float s) { return rsqrtf(s); }
__device__ __forceinline__ double rsqrt_t(double s) { return 1.0 / sqrt(s); }

template <typename T>
__device__ __forceinline__ T dphi(int reg, T t, T g, T ig)
{
    if (reg == 0) return fabs(t) <= g ? t * ig : (t > T(0) ? T(1) : T(-1));
    if (reg == 1) return t * rsqrt_t(t * t + g * g);
    return t;
}

template <typename T>
__device__ __forceinline__ T ddphi(int reg, T t, T g, T ig)
{
    if (reg == 0) return fabs(t) <= g ? ig : T(0);
    if (reg == 1) { const T s = t * t + g * g; const T rs = rsqrt_t(s); return g * g * rs * rs * rs; }
    return T(1);
}

// ------------------------------------------------------------ launch records

enum Mode : int {
    M_APPLY_B = 0, M_APPLY_BT, M_GRAD_LOWER, M_HESS_VEC, M_LOWER_SOLVE, M_UPPER_LOSS,
    M_HYPERGRAD, M_CROSS, M_MAID, M_IMPORT_Y, M_WAIT_SELFTEST
};

struct MaidIn {
    double eps, delta, step, lambda, rho_up, rho_down, nu_up, nu_down, L_gx, eps_stop;
    int max_bt, max_rounds, ll_max_iters, cg_max_iters, k;
    int halted;       // device-resident runs: a step exhausted its rounds, later steps do nothing
};

// Running totals of a device-resident MAID run (not cleared between launches).
struct MaidTotals {
    long long fused_iters;   // FISTA + CG iterations
    long long conv_passes;
    long long upper_iters;   // steps that ran (stop rule not yet fired)
    long long accepted;
};

// Workspace buffers: one padded image each (see Ctx).  The first NBUF_LOWER
// are all a lower-level solve touches (the allocation-free entry holds only
// those).
enum Buf : int {
    B_Y = 0,            // the data y^delta
    B_X0, B_X1,         // FISTA x_k, x_{k+1}
    B_Y0, B_Y1,         // FISTA y_k, y_{k+1}
    B_U,                // residual B x - y, or B p in CG
    B_XK,               // lower-level solution x~
    NBUF_LOWER,
    B_V = NBUF_LOWER,   // A x - y, or B x - y in the kernel gradient
    B_G,                // grad g
    B_R, B_P0, B_P1, B_HP, B_Q,   // CG
    B_XT,               // backtracking trial solution
    B_IN1,              // an imported input image
    NBUF
};

// Launch record of one problem.  Images live in a padded layout: channel c,
// row i, column j of buffer b sit at ws[((b*C + c)*Hp + i + Gy)*Wp + j + Gx],
// and the Gy rows / Gx columns around each image hold its periodic copies
// (ghosts), kept current by every writer.  Any strip's halo tile is then one
// TMA box.  Gx is a multiple of 4 (16-byte aligned boxes) and at least the
// halo width in columns, Gy the halo width in rows.
template <typename T>
struct Ctx {
    CUtensorMap map_s, map_1, map_i;   // boxes: stage (BW x NX), halo-1 tile (40 x MR+2), interior (32 x MR)
    CUtensorMap map_fz;                // FFT path: fzh as FP32 [C*H][W] (box 2 fcb2 x min(H, 256))
    int C, H, W, K, r, Kp;             // Kp: kernel rows padded to a multiple of the stage height PC
    int r4, Gx, Gy, Wp, Hp;            // halo column origin step, ghost widths, padded sizes
    int BW;                            // stage box width: columns col0 - r4 .. col0 - r4 + BW - 1
    int nx, ny, nstrips;               // strips: nx per row band, ny bands per channel
    int wsm;                           // 1: kernel weights in shared memory, 0: in wg (read through L1)
    int multiwrap;                     // 1 when 2Gx > W or 2Gy > H (a pixel may have several copies per axis)
    long long N, HW, HWp, Np;          // dense and padded sizes (Np = C*Hp*Wp per buffer)
    long long *trace;                  // optional: barrier timestamps of CTA 0 (arrive, leave)
    int trace_cap;
    int reg;
    double alpha, rp, beta, w0, ddphi_max;
    T alphaT, rpT, irpT;               // alpha, the regulariser parameter and its reciprocal
    T *ws;                             // padded images (NBUF, or NBUF_LOWER for the lower solve alone)
    T *wg;                             // two slots of both kernel orientations, 2 x 2 x C x K x Kp
    const T *a;                        // kernel of A (library copy)
    T *BT, *ZK;                        // kernels
    double *part;                      // NSLOT x grid
    double *zpart;                     // (grid * warps) x C*K*K
    unsigned *bar;                     // barrier arrival counter
    DevOut *out;
    MaidTotals *totals;                // optional running totals (device-resident runs)
    long long timeout_ns;
    // FFT operator path (FP32 problems with power-of-two H and W; fft = 0: direct)
    int fft, flogH, flogW, fcb, frb;   // log2 H, log2 W, columns per column block, rows per row batch
    float2 *fz, *fs, *fy;              // complex scratch image, kernel spectrum, second spectrum; C x H x W each
    T *fout;                           // the correlation of the last FFT pass, dense C x H x W
    T *fc;                             // B^T y_delta of the current lower solve (FFT path), dense
    const float2 *ftwH, *ftwW;         // twiddles exp(-2 pi i j / n), j < n/2, for n = H and n = W
    // real-to-complex pipeline of the FFT-path FISTA iteration (fr2c = 0: the
    // complex pipeline above carries it)
    int fr2c;                          // 1: lower solves use the real-to-complex pipeline
    int frp;                           // row pairs per row task
    int fcb2;                          // half-spectrum columns per column task
    int fpsh;                          // padding shift of the row tasks' transform slots
    int fnst, fstage, fcstage;         // half-spectrum row stages (1 or 2); floats per row stage; float2 per column stage
    int fncs;                          // column stages (1 or 2)
    int frows;                         // floats of the row tasks' image-row buffer
    float2 *fzh, *fzn;                 // half spectra C x H x W/2 (columns 0 .. W/2-1) and the column W/2, C x H
    float *fsh, *fsn;                  // |F(k)|^2 at those columns: tiled per column task, and at W/2
};

template <typename T>
struct Job {
    int mode;
    const T *b;       // kernel used by the operator
    const T *x;       // image input (dense, caller's)
    T *xo;            // image output (dense, caller's)
    const T *v;       // second image input (Hessian direction, rhs, or q) (dense)
    T *q;             // CG iterate in/out (dense)
    T *z;             // kernel output
    T *bio;           // MAID: kernel in/out
    const T *y;       // data to import first (allocation-free lower solve), or null
    MaidIn *maid_home; // MAID: where the updated state is written back (device-resident runs), or null
    double eps, delta;
    int max_iters, flag;
    int max_steps;    // MAID: upper iterations in this launch (<= 1: one)
    MaidIn maid;
};

// Shared-memory footprint (elements of T) of one CTA with nw warps: both
// kernel orientations when wsm, then per warp two stage buffers (NX = PC + MR
// - 1 rows x BW columns), two halo-1 tiles (MR+2 rows x 40), an interior tile
// (MR x 32) and two mbarriers, each region starting on a 32-element boundary
// (TMA destinations).
template <typename T>
struct Layout {
    int r, r4, Kp, BW, NX, stage, tile1, tileI, w_elems, warp_elems, total;
    __host__ __device__ Layout(int C, int K, int nw, int wsm, bool fft = false)
    {
        constexpr int MR = Cfg<T>::MR, PC = Cfg<T>::PC;
        r = (K - 1) / 2;
        r4 = round_up(r, 4);
        Kp = round_up(K, PC);
        BW = round_up(32 + r + r4, 4);
        NX = PC + MR - 1;
        stage = fft ? 0 : round_up(NX * BW, 32);   // the FFT-path kernel has no correlation stages
        tile1 = round_up((MR + 2) * 40, 32);
        tileI = round_up(MR * 32, 32);
        w_elems = wsm ? round_up(2 * C * Kp * K, 32) : 0;
        warp_elems = 2 * stage + 2 * tile1 + tileI + 32;   // 32: the mbarriers
        total = w_elems + nw * warp_elems;
    }
};

// Bytes of both kernel orientations kept in shared memory at most; larger
// kernels stay in global memory so that shared memory holds eight warps' stages.
constexpr int WSMEM_MAX_BYTES = 40 * 1024;

// Geometry of a problem's padded layout and strips (host and device agree).
struct Geom {
    int r, r4, Gx, Gy, Wp, Hp, Kp, BW, nx, ny, nstrips, wsm, multiwrap;
    long long HW, HWp, N, Np;
};

template <typename T>
inline Geom make_geom(int C, int H, int W, int K)
{
    constexpr int MR = Cfg<T>::MR, PC = Cfg<T>::PC;
    Geom g;
    g.r = (K - 1) / 2;
    g.r4 = round_up(g.r, 4);
    g.Gx = g.r4 > 4 ? g.r4 : 4;
    g.Gy = g.r > 1 ? g.r : 1;
    g.Wp = round_up(W + 2 * g.Gx, 4);
    g.Hp = H + 2 * g.Gy;
    g.Kp = round_up(K, PC);
    g.BW = round_up(32 + g.r + g.r4, 4);
    g.nx = (W + 31) / 32;
    g.ny = (H + MR - 1) / MR;
    g.nstrips = C * g.nx * g.ny;
    g.wsm = (long long)2 * C * K * g.Kp * (long long)sizeof(T) <= WSMEM_MAX_BYTES ? 1 : 0;
    g.multiwrap = (2 * g.Gx > W || 2 * g.Gy > H) ? 1 : 0;
    g.HW = (long long)H * W;
    g.HWp = (long long)g.Hp * g.Wp;
    g.N = g.HW * C;
    g.Np = g.HWp * C;
    return g;
}

// Encodes the three tensor maps of a padded workspace of nbuf images (host
// side, through the driver's cuTensorMapEncodeTiled); 0 on success.
int encode_tensor_maps(void *ws, int nbuf, int C, const Geom &g, int esize, int MR, int NX, CUtensorMap *map_s,
                       CUtensorMap *map_1, CUtensorMap *map_i, char *err, int errlen);


} // namespace adp
