// Device building blocks of libadp: tile geometry, halo loaders, the
// register-blocked direct correlation, deterministic FP64 reductions and the
// bounded grid barrier, plus the launch records (Ctx, Job) shared with the host
// code in adp.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace adp {

constexpr int NW = 4;              // warps per CTA
constexpr int NT = 32 * NW;        // threads per CTA
constexpr int MAXC = 64;           // channels supported (per-channel step cache)
constexpr int KMAX = 63;           // largest odd kernel size supported
constexpr int NSLOT = 8;           // scalar reduction slots

// Rows of outputs per thread: each warp owns a 32-column x MR-row strip, the
// CTA stacks NW strips, so a tile is 32 x (MR*NW).
template <typename T> struct Cfg;
template <> struct Cfg<float>  { static constexpr int MR = 8; };
template <> struct Cfg<double> { static constexpr int MR = 4; };

// Status words shared with the host (values equal adp_status).
enum : int { ST_OK = 0, ST_NONFINITE = 4, ST_NOCONV = 5, ST_LSFAIL = 6, ST_TIMEOUT = 7 };

// Written by the device, copied to pinned host memory after each launch.
struct DevOut {
    int status;
    int iters, cg_iters, capped;
    double gradnorm, resnorm, loss, gradx_norm, znorm, psi;
    // MAID report and updated state
    int accepted, rounds, trials, ll_iters, ll_capped, cg_capped, k, pad;
    double eps, delta, step;
    long long conv_passes;       // number of full-image convolution passes executed
};

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

__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *(const volatile int *)p;
}

// Grid-wide barrier for a cooperative launch.  Thread 0 of each CTA arrives on
// a counter; the last arrival resets it and bumps the generation word the
// others spin on.  Every spin is bounded: after timeout_ns, or as soon as any
// CTA has raised a status, the waiter records ST_TIMEOUT (if nothing else was
// recorded) and returns false, and the caller unwinds.  The host clears the two
// words before every launch.
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *status, long long timeout_ns, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned *count = bar, *gen = bar + 1;
        const unsigned g = ld_acquire_u32(gen);
        __threadfence();
        const unsigned prev = atom_add_acqrel_u32(count, 1u);
        if (prev == gridDim.x - 1) {
            *(volatile unsigned *)count = 0u;
            __threadfence();
            st_release_u32(gen, g + 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (ld_acquire_u32(gen) == g) {
                if ((++spins & 63u) == 0u) {
                    if (ld_volatile_i32(status) != ST_OK) { ok = 0; break; }
                    if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
                        atomicCAS(status, ST_OK, ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        if (ok && ld_volatile_i32(status) != ST_OK) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Sum over a warp; lane 0 holds the result (fixed tree order).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic CTA sum; every thread returns the same value.  `red` is a
// shared array of NW doubles.
__device__ __forceinline__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += red[w];
    return t;
}

// Sum of part[0..n) in a fixed order, computed by every CTA identically (the
// values come from other CTAs, so they are read through L2).
__device__ __forceinline__ double grid_total(const double *part, int n, double *bcast)
{
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < n; i += 32) v += __ldcg(part + i);
        v = warp_sum(v);
        if (threadIdx.x == 0) *bcast = v;
    }
    __syncthreads();
    return *bcast;
}

// Fill s[ii*pitch + jj] (ii < rows, jj < cols <= 128) with f(global index of
// pixel (wrap(r0+ii), wrap(c0+jj)) of the channel starting at cbase).
template <typename T, typename F>
__device__ __forceinline__ void load_tile(T *s, int pitch, int rows, int cols, int H, int W,
                                          long long cbase, int r0, int c0, F f)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int gj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) gj[u] = wrapi(c0 + lane + 32 * u, W);
    for (int ii = warp; ii < rows; ii += NW) {
        const long long rowbase = cbase + (long long)wrapi(r0 + ii, H) * W;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int jj = lane + 32 * u;
            if (jj < cols) s[ii * pitch + jj] = f(rowbase + gj[u]);
        }
    }
}

// Register-blocked direct correlation of one 1 x MR output strip:
//   acc[m] += sum_{p<K, q<K} w[p*K + q] * s[(li0 + m + p)*pitch + lj + q]
// For each kernel column q the MR-row window slides down the column through a
// ring of registers: one new shared load and one broadcast weight per MR FMAs.
template <typename T, int MR>
__device__ __forceinline__ void corr_strip(const T *__restrict__ s, int pitch, const T *__restrict__ w,
                                           int K, int li0, int lj, T (&acc)[MR])
{
    for (int q = 0; q < K; ++q) {
        const T *col = s + li0 * pitch + lj + q;
        const T *wq = w + q;
        T ring[MR];
#pragma unroll
        for (int m = 0; m < MR - 1; ++m) ring[m] = col[m * pitch];
        int p0 = 0;
        for (; p0 + MR <= K; p0 += MR) {
#pragma unroll
            for (int u = 0; u < MR; ++u) {
                ring[(MR - 1 + u) % MR] = col[(p0 + u + MR - 1) * pitch];
                const T wv = wq[(p0 + u) * K];
#pragma unroll
                for (int m = 0; m < MR; ++m) acc[m] = fma(wv, ring[(m + u) % MR], acc[m]);
            }
        }
#pragma unroll
        for (int u = 0; u < MR; ++u) {
            if (p0 + u < K) {
                ring[(MR - 1 + u) % MR] = col[(p0 + u + MR - 1) * pitch];
                const T wv = wq[(p0 + u) * K];
#pragma unroll
                for (int m = 0; m < MR; ++m) acc[m] = fma(wv, ring[(m + u) % MR], acc[m]);
            }
        }
    }
}

// phi' and phi'' of the regularisers (reg: 0 Huber, 1 sqrt, 2 quadratic).
template <typename T>
__device__ __forceinline__ T dphi(int reg, T t, T g)
{
    if (reg == 0) return fabs(t) <= g ? t / g : (t > T(0) ? T(1) : T(-1));
    if (reg == 1) return t / sqrt(t * t + g * g);
    return t;
}

template <typename T>
__device__ __forceinline__ T ddphi(int reg, T t, T g)
{
    if (reg == 0) return fabs(t) <= g ? T(1) / g : T(0);
    if (reg == 1) { const T s = t * t + g * g; return g * g / (s * sqrt(s)); }
    return T(1);
}

// ------------------------------------------------------------ launch records

enum Mode : int {
    M_APPLY_B = 0, M_APPLY_BT, M_GRAD_LOWER, M_HESS_VEC, M_LOWER_SOLVE, M_UPPER_LOSS,
    M_HYPERGRAD, M_CROSS, M_MAID
};

struct MaidIn {
    double eps, delta, step, lambda, rho_up, rho_down, nu_up, nu_down, L_gx;
    int max_bt, max_rounds, ll_max_iters, cg_max_iters, k;
};

template <typename T>
struct Ctx {
    int C, H, W, K, r, h;          // h = max(r, 1)
    int TH, tiles_x, tiles_y, ntiles;
    long long N, HW;
    int reg;
    double alpha, rp, beta, w0, ddphi_max;
    const T *y, *a;                // data and the kernel of A (library copies)
    T *X0, *X1, *X2, *U, *V, *G, *R, *P, *HP, *XT;   // images
    T *BT, *ZK;                    // kernels
    double *part;                  // NSLOT x grid
    double *zpart;                 // grid x C*K*K
    unsigned *bar;                 // barrier words {count, generation}
    DevOut *out;
    long long timeout_ns;
};

template <typename T>
struct Job {
    int mode;
    const T *b;       // kernel used by the operator
    const T *x;       // image input
    T *xo;            // image output
    const T *v;       // second image input (Hessian direction, rhs, or q)
    T *q;             // CG iterate in/out
    T *z;             // kernel output
    T *bio;           // MAID: kernel in/out
    double eps, delta;
    int max_iters, flag;
    MaidIn maid;
};

} // namespace adp
