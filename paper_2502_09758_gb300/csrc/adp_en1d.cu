// 1D elastic-net variant of ADP-beta (Sec. 4.1) on one thread-block cluster.
//
// The operator is a full n x n matrix B, learned with beta = 0: the upper
// level is l(B) = ||A x(B) - y||^2 and the lower level
// h(x; B) = 1/2 ||B x - y||^2 + a1 ||x||_1 + a2 ||x||_2^2 is solved by proximal
// gradient with step lam (Sec. 4.1).  The lower-level accuracy is the norm of
// the proximal-gradient mapping G(x) = (x - prox(x - lam B^T(B x - y))) / lam;
// the hypergradient (Algorithm 1, steps 2-3) solves (B^T B + 2 a2 I)_SS q_S =
// grad g(x)_S on the support S of x by CG and is z = -((B x - y) q^T + (B q) x^T);
// Algorithm 2 (MAID) runs on top with the 2D problem's line search.
//
// Layout: a cluster of P CTAs.  For each operator the solves use (B, or a
// trial of the line search), CTA k forms rows k*m .. k*m+m-1 (m = n/P) of the
// Gram matrix M = B^T B and of c = B^T y in shared memory, so a lower-level
// iteration is one product: grad f(x) = M x - c on this CTA's entries, x+ into
// every CTA's copy of x through distributed shared memory, one cluster barrier.
// Every reduction is summed per CTA, its P partials broadcast and summed in the
// same order everywhere, so every CTA takes every branch identically.  The
// trial operators are never stored: B - alpha z = B + alpha (u q^T + w x^T) is
// formed while tiles of the current B stream through shared memory for M.
#include "adp.h"

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

namespace cg = cooperative_groups;

namespace adp {
void record_error(const char *msg);   // adp.cu: the message adp_last_error returns
} // namespace adp

namespace {

constexpr int P = 8;        // CTAs per cluster
constexpr int NT = 256;     // threads per CTA
constexpr int NW = NT / 32;
constexpr int NPART = 4;    // rotating partial-sum buffers
constexpr int TB = 16;      // rows of B per tile while M forms
constexpr int RB = 2;       // 4 x 4 output blocks of M per thread and pass

enum Mode : int { M_LOWER = 0, M_UPPER, M_HYPER, M_MAID };

struct Out {
    int iters, capped, steps, pad;
    double gn, loss, gxn, res;
};

struct Job {
    int mode, n, max_iters, max_steps;
    double a1, a2, lam, eps, delta;
    const float *A, *AT, *y;
    float *B;                 // operator (read; written on an accepted MAID step)
    float *x;                 // lower-level variable (in/out)
    float *q, *z;             // hypergradient outputs
    adp_maid_state *st;       // MAID state (device copy)
    Out *out;
};

size_t smem_bytes(int n)
{
    const int m = n / P;
    const size_t fl = (size_t)m * n + (size_t)TB * n + 9 * (size_t)n + 5 * (size_t)m;
    return ((fl * 4 + 15) / 16) * 16 + (size_t)(NPART * P + NW) * 8;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

struct En {
    cg::cluster_group cl;
    int k, n, m, r0, lane, warp, pr;
    double a1, a2, lam, ilam;
    float thr, shrink, flam;   // prox constants: lam a1, 1 / (1 + 2 lam a2), lam
    const float *A, *AT, *y;
    float *Mrow, *tile, *x, *xn, *rv, *u, *w, *qf, *pf, *xb, *tC, *gC, *rC, *hC, *yR, *cC;
    double *part, *red;

    __device__ En(const Job &jb, unsigned char *smem) : cl(cg::this_cluster())
    {
        k = (int)cl.block_rank();
        n = jb.n;
        m = n / P;
        r0 = k * m;
        lane = threadIdx.x & 31;
        warp = threadIdx.x >> 5;
        pr = 0;
        a1 = jb.a1;
        a2 = jb.a2;
        lam = jb.lam;
        ilam = 1.0 / lam;
        thr = (float)(lam * a1);
        shrink = (float)(1.0 / (1.0 + 2.0 * lam * a2));
        flam = (float)lam;
        A = jb.A;
        AT = jb.AT;
        y = jb.y;
        float *f = reinterpret_cast<float *>(smem);
        Mrow = f; f += (size_t)m * n;
        tile = f; f += (size_t)TB * n;
        x = f; f += n;
        xn = f; f += n;
        rv = f; f += n;
        u = f; f += n;
        w = f; f += n;
        qf = f; f += n;
        pf = f; f += n;
        xb = f; f += n;
        tC = f; f += n;                               // a slice's new values before their broadcast
        gC = f; f += m;
        rC = f; f += m;
        hC = f; f += m;
        yR = f; f += m;                               // this CTA's entries of y
        cC = f; f += m;                               // ... and of c = B^T y
        for (int i = threadIdx.x; i < m; i += blockDim.x) yR[i] = y[r0 + i];
        size_t off = (size_t)(reinterpret_cast<unsigned char *>(f) - smem);
        off = (off + 15) / 16 * 16;
        part = reinterpret_cast<double *>(smem + off);
        red = part + NPART * P;
    }

    __device__ void csync() { cl.sync(); }

    // value v (held by lane 0) as entry idx of the n-vector buf into every
    // CTA's buf: lane j stores to CTA j (called by the whole warp)
    __device__ void put_all(float *buf, int idx, float v)
    {
        v = __shfl_sync(0xffffffffu, v, 0);
        if (lane < P) cl.map_shared_rank(buf, lane)[idx] = v;
    }

    // deterministic CTA sum (every thread gets the same value)
    __device__ double block_sum(double v)
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double t = 0.0;
        for (int i = 0; i < NW; ++i) t += red[i];
        return t;
    }

    // the cluster total of the CTA values v (a cluster barrier; the same bits in every CTA)
    __device__ double cluster_sum(double v)
    {
        const double t = block_sum(v);
        double *buf = part + pr * P;
        if (threadIdx.x == 0)
            for (int j = 0; j < P; ++j) cl.map_shared_rank(buf, j)[k] = t;
        csync();
        double s = 0.0;
        for (int j = 0; j < P; ++j) s += buf[j];
        pr = (pr + 1) % NPART;
        return s;
    }

    // dot of row il of M (pitch) with the n-vector v: the total in lane 0
    __device__ float row_dot(const float *M, int pitch, int il, const float *v) const
    {
        float s = 0.f;
        const float *row = M + (size_t)il * pitch;
        for (int j = lane; j < n; j += 32) s = fmaf(row[j], v[j], s);
        return warp_sum_f(s);
    }

    // this CTA's rows of M = Bt^T Bt and of c = Bt^T y for the operator
    // Bt = B (al = 0) or the trial Bt = B + al (uu qq^T + ww xx^T) of the line
    // search: tiles of TB rows of Bt through shared memory, each thread
    // accumulating 4 x 4 blocks of M (rows in its warp's block, consecutive
    // columns across lanes), the sums over the rows of B in order
    __device__ void form_M(const float *B, float al, const float *uu, const float *qq, const float *ww,
                           const float *xx)
    {
        const int nk = n >> 2, nblk = (m >> 2) * nk;
        for (int b0 = 0; b0 < nblk; b0 += NT * RB) {
            float acc[RB][16];
            int jb[RB], kb[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int bb = b0 + threadIdx.x + r * NT;
                jb[r] = bb < nblk ? bb / nk : -1;
                kb[r] = bb < nblk ? bb - (bb / nk) * nk : 0;
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[r][q] = 0.f;
            }
            float cacc = 0.f;
            const bool cthr = b0 == 0 && threadIdx.x < m;
            for (int i0 = 0; i0 < n; i0 += TB) {
                const int rows = n - i0 < TB ? n - i0 : TB;
                __syncthreads();                      // the previous tile is consumed
                for (int e = threadIdx.x; e < rows * n; e += NT) {
                    const int ii = e / n, j = e - ii * n, i = i0 + ii;
                    float v = B[(size_t)i * n + j];
                    if (al != 0.f) v = fmaf(al, fmaf(uu[i], qq[j], ww[i] * xx[j]), v);
                    tile[e] = v;
                }
                __syncthreads();
                for (int ii = 0; ii < rows; ++ii) {
                    const float *tr = tile + (size_t)ii * n;
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        if (jb[r] < 0) continue;
                        const float4 av = *reinterpret_cast<const float4 *>(tr + r0 + 4 * jb[r]);
                        const float4 bv = *reinterpret_cast<const float4 *>(tr + 4 * kb[r]);
                        const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                        for (int p = 0; p < 4; ++p)
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[r][4 * p + q] = fmaf(a4[p], b4[q], acc[r][4 * p + q]);
                    }
                    if (cthr) cacc = fmaf(tr[r0 + threadIdx.x], yfull(i0 + ii), cacc);
                }
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (jb[r] < 0) continue;
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    *reinterpret_cast<float4 *>(Mrow + (size_t)(4 * jb[r] + p) * n + 4 * kb[r]) =
                        make_float4(acc[r][4 * p], acc[r][4 * p + 1], acc[r][4 * p + 2], acc[r][4 * p + 3]);
            }
            if (cthr) cC[threadIdx.x] = cacc;
        }
        __syncthreads();
    }
    __device__ float yfull(int i) const { return __ldg(y + i); }

    // rows r0 .. r0+m-1 of Bt (= B + al (uu qq^T + ww xx^T)) times v, from global
    // memory: the total of row il in lane 0
    __device__ float brow_dot(const float *B, float al, const float *uu, const float *qq, const float *ww,
                              const float *xx, int il, const float *v) const
    {
        const int i = r0 + il;
        const float *row = B + (size_t)i * n;
        float s = 0.f;
        for (int j = lane; j < n; j += 32) {
            float bv = __ldg(row + j);
            if (al != 0.f) bv = fmaf(al, fmaf(uu[i], qq[j], ww[i] * xx[j]), bv);
            s = fmaf(bv, v[j], s);
        }
        return warp_sum_f(s);
    }

    __device__ float prox(float v) const
    {
        const float s = fmaxf(fabsf(v) - thr, 0.f);
        return copysignf(s, v) * shrink;
    }

    // proximal gradient on the member vector x (in place, possibly after
    // buffer swaps): returns updates made, gn = ||G|| of the returned iterate
    __device__ int lower(double eps, int max_iters, double &gn)
    {
        int it = 0;
        for (;;) {
            // x+ = prox(x - lam (M x - c)) on this CTA's entries, into every CTA;
            // G = (x - x+) / lam
            double gl = 0.0;
            for (int jl = warp; jl < m; jl += NW) {
                const float s = row_dot(Mrow, n, jl, x) - cC[jl];
                const float xc = x[r0 + jl];
                const float xp = prox(xc - flam * s);
                put_all(xn, r0 + jl, xp);
                if (lane == 0) {
                    const double G = ((double)xc - (double)xp) * ilam;
                    gl += G * G;
                }
            }
            gn = sqrt(cluster_sum(gl));
            if (gn <= eps || it >= max_iters) return it;
            float *t = x;
            x = xn;
            xn = t;
            ++it;
        }
    }

    // l = ||A xv - y||^2 and ||grad g||; grad g's slice on this CTA's
    // columns into gC.  rv is overwritten with A xv - y.
    __device__ void upper(const float *xv, double &loss, double &gxn)
    {
        double le = 0.0;
        for (int il = warp; il < m; il += NW) {
            float s = 0.f;
            const float *row = A + (size_t)(r0 + il) * n;
            for (int j = lane; j < n; j += 32) s = fmaf(__ldg(row + j), xv[j], s);
            s = warp_sum_f(s);
            const float e = s - yR[il];
            put_all(rv, r0 + il, e);
            if (lane == 0) le += (double)e * (double)e;
        }
        loss = cluster_sum(le);
        double lg = 0.0;
        for (int jl = warp; jl < m; jl += NW) {
            float s = 0.f;
            const float *row = AT + (size_t)(r0 + jl) * n;
            for (int i = lane; i < n; i += 32) s = fmaf(__ldg(row + i), rv[i], s);
            s = warp_sum_f(s);
            if (lane == 0) {
                gC[jl] = 2.f * s;
                lg += (double)gC[jl] * (double)gC[jl];
            }
        }
        gxn = sqrt(cluster_sum(lg));
    }

    // Algorithm 1, steps 2-3, at the member x (its gradient slice in gC from
    // upper, M of the operator B in Mrow): CG on the support; q in qf,
    // u = B x - y in u, w = B q in w (all full, B's rows read from global
    // memory); returns iterations; zz = ||z||^2
    __device__ int hyper(const float *B, double delta, int max_iters, double &res, double &zz)
    {
        double rl = 0.0;
        for (int jl = threadIdx.x; jl < m; jl += NT) {
            const float r = x[r0 + jl] != 0.f ? gC[jl] : 0.f;
            rC[jl] = r;
            hC[jl] = 0.f;                             // q's slice
            rl += (double)r * (double)r;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < P * m; e += NT) {   // p = r into every CTA
            const int j = e / m, jl = e - j * m;
            cl.map_shared_rank(pf, j)[r0 + jl] = rC[jl];
        }
        double rr = cluster_sum(rl);
        int it = 0;
        while (sqrt(rr) > delta && it < max_iters) {
            double pl = 0.0;
            for (int jl = warp; jl < m; jl += NW) {   // H p = M p + 2 a2 p on this CTA's entries of S
                const float s = row_dot(Mrow, n, jl, pf);
                if (lane == 0) {
                    const float pc = pf[r0 + jl];
                    const float hp = x[r0 + jl] != 0.f ? fmaf((float)(2.0 * a2), pc, s) : 0.f;
                    u[r0 + jl] = hp;                  // local scratch: H p's slice
                    pl += (double)pc * (double)hp;
                }
            }
            const double php = cluster_sum(pl);
            if (!(php > 0.0)) break;
            const float al = (float)(rr / php);
            double nl = 0.0;
            for (int jl = threadIdx.x; jl < m; jl += NT) {
                hC[jl] = fmaf(al, pf[r0 + jl], hC[jl]);
                const float r = fmaf(-al, u[r0 + jl], rC[jl]);
                rC[jl] = r;
                nl += (double)r * (double)r;
            }
            const double rn = cluster_sum(nl);
            const float be = (float)(rn / rr);
            for (int jl = threadIdx.x; jl < m; jl += NT) tC[jl] = fmaf(be, pf[r0 + jl], rC[jl]);
            __syncthreads();                          // the old slice is read before any copy lands
            for (int e = threadIdx.x; e < P * m; e += NT) {
                const int j = e / m, jl = e - j * m;
                cl.map_shared_rank(pf, j)[r0 + jl] = tC[jl];
            }
            csync();
            rr = rn;
            ++it;
        }
        res = sqrt(rr);
        // q into every CTA, then u = B x - y and w = B q by rows into every CTA
        for (int e = threadIdx.x; e < P * m; e += NT) {
            const int j = e / m, jl = e - j * m;
            cl.map_shared_rank(qf, j)[r0 + jl] = hC[jl];
        }
        csync();
        for (int il = warp; il < m; il += NW) {
            const float s1 = brow_dot(B, 0.f, nullptr, nullptr, nullptr, nullptr, il, x);
            const float s2 = brow_dot(B, 0.f, nullptr, nullptr, nullptr, nullptr, il, qf);
            put_all(u, r0 + il, s1 - yR[il]);
            put_all(w, r0 + il, s2);
        }
        csync();
        double zl = 0.0;
        for (int e = threadIdx.x; e < m * n; e += NT) {
            const int il = e / n, j = e - il * n, i = r0 + il;
            const double v = (double)u[i] * qf[j] + (double)w[i] * x[j];
            zl += v * v;
        }
        zz = cluster_sum(zl);
        return it;
    }

    __device__ void copy_vec(float *dst, const float *src)
    {
        for (int i = threadIdx.x; i < n; i += NT) dst[i] = src[i];
        __syncthreads();
    }
};

// One MAID step (Algorithm 2, the same control as adp_maid_step) on the
// state s (registers, identical in every thread); B and x in global memory.
__device__ bool maid_step(En &e, const Job &jb, adp_maid_state &s)
{
    s.accepted = s.rounds = s.trials = s.ll_iters = s.cg_iters = 0;
    s.ll_capped = s.cg_capped = s.stopped = 0;
    if (s.eps_stop > 0.0 && s.eps <= s.eps_stop) {
        s.stopped = 1;
        return false;
    }
    e.form_M(jb.B, 0.f, nullptr, nullptr, nullptr, nullptr);
    for (int i = threadIdx.x; i < e.n; i += NT) e.x[i] = jb.x[i];
    __syncthreads();
    int j = s.max_bt;
    for (int round = 0; round < s.max_rounds; ++round, ++j) {
        s.rounds = round + 1;
        double gn;
        s.ll_iters += e.lower(s.eps, s.ll_max_iters, gn);
        if (gn > s.eps) s.ll_capped = 1;
        double l0, gx0;
        e.upper(e.x, l0, gx0);
        double res, zz;
        const int cit = e.hyper(jb.B, s.delta, s.cg_max_iters, res, zz);
        s.cg_iters += cit;
        if (res > s.delta) s.cg_capped = 1;
        s.znorm = sqrt(zz);
        e.copy_vec(e.xb, e.x);                        // x~(b_k): the trials' warm start
        for (int i = 0; i < j; ++i) {
            s.trials += 1;
            e.form_M(jb.B, (float)s.step, e.u, e.qf, e.w, e.xb);
            e.copy_vec(e.x, e.xb);
            e.csync();
            s.ll_iters += e.lower(s.eps, s.ll_max_iters, gn);
            if (gn > s.eps) s.ll_capped = 1;
            double l1, gx1;
            e.upper(e.x, l1, gx1);
            const double eb = s.eps;                  // eps_bar_{k+1} = eps_k
            const double psi = l1 + gx1 * eb + 0.5 * s.L_gx * eb * eb - l0 + gx0 * eb + s.lambda * s.step * zz;
            s.psi = psi;
            if (psi <= 0.0) {
                // b_{k+1}: this CTA's rows of the trial operator, and x~(b_{k+1})
                e.csync();                            // every CTA has formed its M from B
                const float al = (float)s.step;
                for (int q = threadIdx.x; q < e.m * e.n; q += NT) {
                    const int il = q / e.n, jj = q - il * e.n, i = e.r0 + il;
                    float *bp = jb.B + (size_t)i * e.n + jj;
                    *bp = fmaf(al, fmaf(e.u[i], e.qf[jj], e.w[i] * e.xb[jj]), *bp);
                }
                if (e.k == 0)
                    for (int q = threadIdx.x; q < e.n; q += NT) jb.x[q] = e.x[q];
                s.loss = l1;
                s.gradx_norm = gx1;
                s.eps *= s.nu_up;
                s.delta *= s.nu_up;
                s.step *= s.rho_up;
                s.k += 1;
                s.accepted = 1;
                e.csync();
                return true;
            }
            s.step *= s.rho_down;
        }
        s.loss = l0;
        s.gradx_norm = gx0;
        s.eps *= s.nu_down;
        s.delta *= s.nu_down;
        // the next round starts again from b_k and x~(b_k)
        e.csync();
        e.form_M(jb.B, 0.f, nullptr, nullptr, nullptr, nullptr);
        e.copy_vec(e.x, e.xb);
        e.csync();
        if (s.eps_stop > 0.0 && s.eps <= s.eps_stop) {
            s.stopped = 1;
            break;
        }
    }
    return false;
}

__global__ void __launch_bounds__(NT, 1) en1d_kernel(const __grid_constant__ Job jb)
{
    extern __shared__ __align__(16) unsigned char smem[];
    En e(jb, smem);
    const bool lead = e.k == 0 && threadIdx.x == 0;
    switch (jb.mode) {
    case M_LOWER: {
        e.form_M(jb.B, 0.f, nullptr, nullptr, nullptr, nullptr);
        for (int i = threadIdx.x; i < e.n; i += NT) e.x[i] = jb.x[i];
        e.csync();
        double gn;
        const int it = e.lower(jb.eps, jb.max_iters, gn);
        if (e.k == 0)
            for (int i = threadIdx.x; i < e.n; i += NT) jb.x[i] = e.x[i];
        if (lead) {
            jb.out->iters = it;
            jb.out->gn = gn;
        }
        break;
    }
    case M_UPPER: {
        for (int i = threadIdx.x; i < e.n; i += NT) e.x[i] = jb.x[i];
        e.csync();
        double l, g;
        e.upper(e.x, l, g);
        if (lead) {
            jb.out->loss = l;
            jb.out->gxn = g;
        }
        break;
    }
    case M_HYPER: {
        e.form_M(jb.B, 0.f, nullptr, nullptr, nullptr, nullptr);
        for (int i = threadIdx.x; i < e.n; i += NT) e.x[i] = jb.x[i];
        e.csync();
        double l, g, res, zz;
        e.upper(e.x, l, g);
        const int it = e.hyper(jb.B, jb.delta, jb.max_iters, res, zz);
        for (int q = threadIdx.x; q < e.m * e.n; q += NT) {
            const int il = q / e.n, j = q - il * e.n, i = e.r0 + il;
            jb.z[(size_t)i * e.n + j] = -fmaf(e.u[i], e.qf[j], e.w[i] * e.x[j]);
        }
        for (int jl = threadIdx.x; jl < e.m; jl += NT) jb.q[e.r0 + jl] = e.qf[e.r0 + jl];
        if (lead) {
            jb.out->iters = it;
            jb.out->res = res;
            jb.out->capped = res > jb.delta;
        }
        break;
    }
    case M_MAID: {
        adp_maid_state s = *jb.st;
        int steps = 0;
        while (steps < jb.max_steps) {
            const bool acc = maid_step(e, jb, s);
            ++steps;
            if (!acc || s.stopped) break;
            e.csync();                                // B and x in global memory for the next step
        }
        e.csync();
        if (lead) {
            *jb.st = s;
            jb.out->steps = steps;
        }
        break;
    }
    default: break;
    }
    e.csync();                                        // no CTA leaves while others read its shared memory
}

__attribute__((format(printf, 1, 2))) void err(const char *fmt, ...)
{
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    adp::record_error(b);
}

#define CKE(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            err("%s (code %lld)", cudaGetErrorString(e_), (long long)e_);                          \
            return ADP_ECUDA;                                                                      \
        }                                                                                          \
    } while (0)

} // namespace

struct adp_en1d {
    adp_en1d_params prm;
    int device;
    cudaStream_t stream;
    const float *A, *y;
    float *AT;                 // A^T (row-major), made at creation
    Out *out_d, *out_h;
    adp_maid_state *st_d, *st_h;
    size_t smem;
    double L_gx;
};

namespace {

adp_status launch(adp_en1d *p, Job jb)
{
    jb.n = p->prm.n;
    jb.a1 = p->prm.a1;
    jb.a2 = p->prm.a2;
    jb.lam = p->prm.lam;
    jb.A = p->A;
    jb.AT = p->AT;
    jb.y = p->y;
    jb.out = p->out_d;
    CKE(cudaSetDevice(p->device));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = p->smem;
    cfg.stream = p->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CKE(cudaLaunchKernelEx(&cfg, en1d_kernel, jb));
    CKE(cudaGetLastError());
    CKE(cudaMemcpyAsync(p->out_h, p->out_d, sizeof(Out), cudaMemcpyDeviceToHost, p->stream));
    CKE(cudaStreamSynchronize(p->stream));
    return ADP_OK;
}

} // namespace

extern "C" {

adp_status adp_en1d_create(const adp_en1d_params *prm, const float *A, const float *y, void *stream, adp_en1d **out)
{
    if (!prm || !A || !y || !out) {
        err("null argument");
        return ADP_EINVAL;
    }
    *out = nullptr;
    if (prm->n < 4 * P || prm->n > ADP_EN1D_MAX_N || prm->n % (4 * P)) {
        err("n must be a multiple of 32 in 32 .. %d", ADP_EN1D_MAX_N);
        return ADP_EINVAL;
    }
    if (!(prm->a1 >= 0.0) || !(prm->a2 >= 0.0) || !(prm->lam > 0.0)) {
        err("a1, a2 must be >= 0 and lam > 0");
        return ADP_EINVAL;
    }
    adp_en1d *p = (adp_en1d *)calloc(1, sizeof(adp_en1d));
    if (!p) {
        err("host allocation failed");
        return ADP_ENOMEM;
    }
    p->prm = *prm;
    p->stream = (cudaStream_t)stream;
    p->A = A;
    p->y = y;
    p->smem = smem_bytes(prm->n);
    const int n = prm->n;
    auto fail = [&](adp_status st) {
        adp_en1d_destroy(p);
        return st;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        err("no current CUDA device");
        return fail(ADP_ECUDA);
    }
    {
        int maxsmem = 0;
        cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
        if ((size_t)maxsmem < p->smem) {
            err("shared memory per CTA too small for n = %d", n);
            return fail(ADP_EINVAL);
        }
        cudaError_t e = cudaFuncSetAttribute(en1d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
        if (e != cudaSuccess) {
            err("%s (code %lld)", cudaGetErrorString(e), (long long)e);
            return fail(ADP_ECUDA);
        }
    }
    if (cudaMalloc((void **)&p->AT, (size_t)n * n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&p->out_d, sizeof(Out)) != cudaSuccess ||
        cudaMalloc((void **)&p->st_d, sizeof(adp_maid_state)) != cudaSuccess ||
        cudaMallocHost((void **)&p->out_h, sizeof(Out)) != cudaSuccess ||
        cudaMallocHost((void **)&p->st_h, sizeof(adp_maid_state)) != cudaSuccess) {
        err("device allocation failed");
        return fail(ADP_ENOMEM);
    }
    // A^T and the bound 2 ||A||_1 ||A||_inf, from a host copy of A
    float *h = (float *)malloc((size_t)n * n * sizeof(float)), *ht = (float *)malloc((size_t)n * n * sizeof(float));
    if (!h || !ht) {
        free(h);
        free(ht);
        err("host allocation failed");
        return fail(ADP_ENOMEM);
    }
    cudaError_t e = cudaMemcpyAsync(h, A, (size_t)n * n * sizeof(float), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        free(h);
        free(ht);
        err("%s (code %lld)", cudaGetErrorString(e), (long long)e);
        return fail(ADP_ECUDA);
    }
    double c1 = 0.0, ci = 0.0;
    for (int i = 0; i < n; ++i) {
        double rs = 0.0, cs = 0.0;
        for (int j = 0; j < n; ++j) {
            ht[(size_t)j * n + i] = h[(size_t)i * n + j];
            rs += fabs((double)h[(size_t)i * n + j]);
            cs += fabs((double)h[(size_t)j * n + i]);
        }
        if (rs > ci) ci = rs;
        if (cs > c1) c1 = cs;
    }
    p->L_gx = 2.0 * c1 * ci;
    e = cudaMemcpyAsync(p->AT, ht, (size_t)n * n * sizeof(float), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    free(h);
    free(ht);
    if (e != cudaSuccess) {
        err("%s (code %lld)", cudaGetErrorString(e), (long long)e);
        return fail(ADP_ECUDA);
    }
    int ncl = 0;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(P, 1, 1);
        cfg.blockDim = dim3(NT, 1, 1);
        cfg.dynamicSmemBytes = p->smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = P;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&ncl, en1d_kernel, &cfg) != cudaSuccess || ncl < 1) {
            err("a cluster of 8 CTAs with this shared memory cannot be resident");
            return fail(ADP_EINVAL);
        }
    }
    *out = p;
    return ADP_OK;
}

void adp_en1d_destroy(adp_en1d *p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->AT) cudaFree(p->AT);
    if (p->out_d) cudaFree(p->out_d);
    if (p->st_d) cudaFree(p->st_d);
    if (p->out_h) cudaFreeHost(p->out_h);
    if (p->st_h) cudaFreeHost(p->st_h);
    free(p);
}

adp_status adp_en1d_lower_solve(adp_en1d *p, const float *B, float *x, double eps, int max_iters, int *iters,
                                double *gmap_norm)
{
    if (!p || !B || !x || max_iters < 0) {
        err("invalid arguments");
        return ADP_EINVAL;
    }
    Job jb = {};
    jb.mode = M_LOWER;
    jb.B = const_cast<float *>(B);
    jb.x = x;
    jb.eps = eps;
    jb.max_iters = max_iters;
    const adp_status st = launch(p, jb);
    if (st != ADP_OK) return st;
    if (iters) *iters = p->out_h->iters;
    if (gmap_norm) *gmap_norm = p->out_h->gn;
    return ADP_OK;
}

adp_status adp_en1d_upper_loss(adp_en1d *p, const float *x, double *loss, double *gradx_norm)
{
    if (!p || !x) {
        err("invalid arguments");
        return ADP_EINVAL;
    }
    Job jb = {};
    jb.mode = M_UPPER;
    jb.x = const_cast<float *>(x);
    const adp_status st = launch(p, jb);
    if (st != ADP_OK) return st;
    if (loss) *loss = p->out_h->loss;
    if (gradx_norm) *gradx_norm = p->out_h->gxn;
    return ADP_OK;
}

adp_status adp_en1d_hypergrad(adp_en1d *p, const float *B, const float *x, double delta, int max_iters, float *q,
                              float *z, int *cg_iters, double *resnorm)
{
    if (!p || !B || !x || !q || !z || max_iters < 0) {
        err("invalid arguments");
        return ADP_EINVAL;
    }
    Job jb = {};
    jb.mode = M_HYPER;
    jb.B = const_cast<float *>(B);
    jb.x = const_cast<float *>(x);
    jb.q = q;
    jb.z = z;
    jb.delta = delta;
    jb.max_iters = max_iters;
    const adp_status st = launch(p, jb);
    if (st != ADP_OK) return st;
    if (cg_iters) *cg_iters = p->out_h->iters;
    if (resnorm) *resnorm = p->out_h->res;
    return ADP_OK;
}

adp_status adp_en1d_maid_init(adp_en1d *p, adp_maid_state *s)
{
    if (!p || !s) {
        err("invalid arguments");
        return ADP_EINVAL;
    }
    memset(s, 0, sizeof *s);
    s->eps = 1e-2;
    s->delta = 1e-2;
    s->step = 0.1;
    s->lambda = 1e-4;
    s->rho_up = 1.1;
    s->rho_down = 0.5;
    s->nu_up = 1.25;
    s->nu_down = 0.5;
    s->L_gx = p->L_gx;
    s->eps_stop = 0.0;
    s->max_bt = 5;
    s->max_rounds = 20;
    s->ll_max_iters = 300;
    s->cg_max_iters = 1000;
    return ADP_OK;
}

static adp_status maid_launch(adp_en1d *p, adp_maid_state *s, float *B, float *x, int max_steps, int *steps)
{
    if (!p || !s || !B || !x || max_steps < 1) {
        err("invalid arguments");
        return ADP_EINVAL;
    }
    *p->st_h = *s;
    CKE(cudaSetDevice(p->device));
    CKE(cudaMemcpyAsync(p->st_d, p->st_h, sizeof *s, cudaMemcpyHostToDevice, p->stream));
    Job jb = {};
    jb.mode = M_MAID;
    jb.B = B;
    jb.x = x;
    jb.st = p->st_d;
    jb.max_steps = max_steps;
    const adp_status st = launch(p, jb);
    if (st != ADP_OK) return st;
    CKE(cudaMemcpyAsync(p->st_h, p->st_d, sizeof *s, cudaMemcpyDeviceToHost, p->stream));
    CKE(cudaStreamSynchronize(p->stream));
    *s = *p->st_h;
    if (steps) *steps = p->out_h->steps;
    return ADP_OK;
}

adp_status adp_en1d_maid_step(adp_en1d *p, adp_maid_state *s, float *B, float *x)
{
    return maid_launch(p, s, B, x, 1, nullptr);
}

adp_status adp_en1d_maid_run(adp_en1d *p, adp_maid_state *s, float *B, float *x, int max_steps, int *steps)
{
    return maid_launch(p, s, B, x, max_steps, steps);
}

} // extern "C"
