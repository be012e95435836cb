// The persistent engine of libadp: every phase of the hot path as a device
// member function and the cooperative kernel that runs one program of phases.
// Included by the per-precision translation units adp_f32.cu and adp_f64.cu.
//
// Convolution geometry (Eq. 2.4): (B x)[c,i,j] = sum_{p,q} b[c,p,q] x[c,i-p+r,j-q+r].
// A tile of 32 x TH outputs loads its input with an r-pixel periodic halo into
// shared memory (origin at (row0-r, col0-r)); then B x is the correlation of the
// tile with the flipped kernel and B^T z the correlation with b itself.
#pragma once

#include "adp_device.cuh"

namespace adp {

template <typename T>
struct Eng {
    const Ctx<T> &cx;
    T *sA, *sB, *sC, *sU, *sV, *sw;
    int pitch;                     // of sA/sB: 32 + 2h
    double *red, *bcast, *tau;
    int *sflag;
    int lane, warp, tid;
    bool alive;                    // false once a barrier gave up

    __device__ Eng(const Ctx<T> &c, unsigned char *smem, double *red_, double *bcast_, double *tau_, int *sflag_)
        : cx(c), red(red_), bcast(bcast_), tau(tau_), sflag(sflag_), alive(true)
    {
        pitch = 32 + 2 * cx.h;
        const int halo_elems = (cx.TH + 2 * cx.h) * pitch;
        const int halo1 = (cx.TH + 2) * 34;
        T *p = reinterpret_cast<T *>(smem);
        sA = p; p += halo_elems;
        sB = p; p += halo_elems;
        sC = p; p += halo1;
        sU = p; p += cx.TH * 32;
        sV = p; p += cx.TH * 32;
        sw = p;
        lane = threadIdx.x & 31;
        warp = threadIdx.x >> 5;
        tid = threadIdx.x;
    }

    __device__ bool sync()
    {
        if (!alive) return false;
        alive = grid_sync(cx.bar, &cx.out->status, cx.timeout_ns, sflag);
        return alive;
    }

    __device__ void fail(int st)
    {
        if (tid == 0) atomicCAS(&cx.out->status, ST_OK, st);
        alive = false;
    }

    __device__ void tile_of(int t, int &c, int &row0, int &col0) const
    {
        const int per = cx.tiles_x * cx.tiles_y;
        c = t / per;
        const int rem = t - c * per;
        const int ty = rem / cx.tiles_x;
        row0 = ty * cx.TH;
        col0 = (rem - ty * cx.tiles_x) * 32;
    }

    // weights of channel c into sw, flipped for B, as stored for B^T
    __device__ void load_w(const T *b, int c, bool flip)
    {
        const int KK = cx.K * cx.K;
        const T *bc = b + (long long)c * KK;
        for (int e = tid; e < KK; e += NT) sw[e] = flip ? __ldcg(bc + (KK - 1 - e)) : __ldcg(bc + e);
    }

    // record the partial of this CTA in a slot and return the grid total after
    // a barrier; all CTAs get identical bits
    __device__ double reduce(double mine, int slot)
    {
        const double cta = block_sum(mine, red);
        if (tid == 0) cx.part[slot * gridDim.x + blockIdx.x] = cta;
        if (!sync()) return 0.0;
        return grid_total(cx.part + slot * gridDim.x, gridDim.x, bcast);
    }

    // ------------------------------------------------------------ conv pass
    // One pass over all tiles: load the halo-r tile from src, correlate with
    // the (flipped) kernel of channel c, and hand each in-image output to epi,
    // whose return values are summed (FP32 per strip, FP64 across strips).
    template <typename Src, typename Pre, typename Epi>
    __device__ double conv_pass(const T *b, bool flip, Src src, Pre pre, Epi epi)
    {
        constexpr int MR = Cfg<T>::MR;
        const int r = cx.r, K = cx.K, H = cx.H, W = cx.W;
        double part = 0.0;
        for (int t = blockIdx.x; t < cx.ntiles; t += gridDim.x) {
            int c, row0, col0;
            tile_of(t, c, row0, col0);
            const long long cbase = (long long)c * cx.HW;
            load_w(b, c, flip);
            load_tile(sA, pitch, cx.TH + 2 * r, 32 + 2 * r, H, W, cbase, row0 - r, col0 - r, src);
            pre(c, row0, col0, cbase);
            __syncthreads();
            T acc[MR];
#pragma unroll
            for (int m = 0; m < MR; ++m) acc[m] = T(0);
            const int li0 = warp * MR;
            corr_strip<T, MR>(sA, pitch, sw, K, li0, lane, acc);
            T s = T(0);
            const int gj = col0 + lane;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int gi = row0 + li0 + m;
                if (gi < H && gj < W) s += epi(c, li0 + m, lane, cbase + (long long)gi * W + gj, acc[m]);
            }
            part += (double)s;
            __syncthreads();
        }
        return part;
    }

    // ------------------------------------------------------------ helpers
    __device__ long long gstride() const { return (long long)gridDim.x * NT; }
    __device__ long long gstart() const { return (long long)blockIdx.x * NT + tid; }

    // 1/L_c for FISTA on channel c with kernel b: L_c = ||b_c||_1^2 + 8 alpha sup phi''
    __device__ void compute_tau(const T *b)
    {
        const int KK = cx.K * cx.K;
        for (int c = 0; c < cx.C; ++c) {
            double s = 0.0;
            for (int e = tid; e < KK; e += NT) s += fabs((double)__ldcg(b + (long long)c * KK + e));
            const double l1 = block_sum(s, red);
            if (tid == 0) tau[c] = 1.0 / (l1 * l1 + 8.0 * cx.alpha * cx.ddphi_max);
        }
        __syncthreads();
    }

    // TV gradient at interior pixel (li, lj) of a halo-1 tile s (pitch 34)
    __device__ T tv_grad(const T *s, int li, int lj) const
    {
        const T g = (T)cx.rp;
        const T yc = s[(li + 1) * 34 + lj + 1];
        const T yl = s[(li + 1) * 34 + lj], yr = s[(li + 1) * 34 + lj + 2];
        const T yu = s[li * 34 + lj + 1], yd = s[(li + 2) * 34 + lj + 1];
        return dphi<T>(cx.reg, yc - yl, g) - dphi<T>(cx.reg, yr - yc, g) +
               dphi<T>(cx.reg, yc - yu, g) - dphi<T>(cx.reg, yd - yc, g);
    }

    // D^T(phi''(D x) . D v) at interior pixel (li, lj); x in sx, v in sv (halo 1)
    __device__ T tv_hess(const T *sx, const T *sv, int li, int lj) const
    {
        const T g = (T)cx.rp;
        const int o = (li + 1) * 34 + lj + 1;
        const T xc = sx[o], vc = sv[o];
        const T wl = ddphi<T>(cx.reg, xc - sx[o - 1], g);
        const T wr = ddphi<T>(cx.reg, sx[o + 1] - xc, g);
        const T wu = ddphi<T>(cx.reg, xc - sx[o - 34], g);
        const T wd = ddphi<T>(cx.reg, sx[o + 34] - xc, g);
        return wl * (vc - sv[o - 1]) - wr * (sv[o + 1] - vc) + wu * (vc - sv[o - 34]) - wd * (sv[o + 34] - vc);
    }

    __device__ void load_halo1(T *s, int row0, int col0, long long cbase, const T *src) const
    {
        load_tile(s, 34, cx.TH + 2, 34, cx.H, cx.W, cbase, row0 - 1, col0 - 1,
                  [=](long long g) { return __ldcg(src + g); });
    }

    // ------------------------------------------------------------ programs
    // out = B x (flip) or B^T x
    __device__ void apply(const T *b, const T *x, T *out, bool transpose)
    {
        conv_pass(b, !transpose, [=](long long g) { return __ldcg(x + g); },
                  [](int, int, int, long long) {},
                  [=](int, int, int, long long g, T v) { out[g] = v; return T(0); });
    }

    // U = B x - y   (first half of grad_x h)
    __device__ void residual(const T *b, const T *x, T *U)
    {
        const T *y = cx.y;
        conv_pass(b, true, [=](long long g) { return __ldcg(x + g); },
                  [](int, int, int, long long) {},
                  [=](int, int, int, long long g, T v) { U[g] = v - __ldg(y + g); return T(0); });
    }

    // grad = B^T U + alpha grad J(x); optional store; returns ||grad||^2 partial
    __device__ double grad_from_residual(const T *b, const T *U, const T *x, T *out)
    {
        const T al = (T)cx.alpha;
        T *sBl = sB;
        return conv_pass(b, false, [=](long long g) { return __ldcg(U + g); },
                         [=](int, int row0, int col0, long long cbase) { load_halo1(sBl, row0, col0, cbase, x); },
                         [=](int, int li, int lj, long long g, T v) {
                             const T gr = v + al * tv_grad(sBl, li, lj);
                             if (out) out[g] = gr;
                             return gr * gr;
                         });
    }

    __device__ void grad_lower(const T *b, const T *x, T *out)
    {
        residual(b, x, cx.U);
        if (!sync()) return;
        const double ss = reduce(grad_from_residual(b, cx.U, x, out), 0);
        if (tid == 0 && blockIdx.x == 0) cx.out->gradnorm = sqrt(ss);
    }

    // out = B^T B v + alpha D^T(phi''(D x) . D v); returns <v, out> partial
    __device__ double hess_vec(const T *b, const T *x, const T *v, T *out)
    {
        const T al = (T)cx.alpha;
        T *U = cx.U;
        conv_pass(b, true, [=](long long g) { return __ldcg(v + g); },
                  [](int, int, int, long long) {},
                  [=](int, int, int, long long g, T val) { U[g] = val; return T(0); });
        if (!sync()) return 0.0;
        T *sBl = sB, *sCl = sC;
        return conv_pass(b, false, [=](long long g) { return __ldcg(U + g); },
                         [=](int, int row0, int col0, long long cbase) {
                             load_halo1(sBl, row0, col0, cbase, x);
                             load_halo1(sCl, row0, col0, cbase, v);
                         },
                         [=](int, int li, int lj, long long g, T val) {
                             const T hv = val + al * tv_hess(sBl, sCl, li, lj);
                             out[g] = hv;
                             return hv * sCl[(li + 1) * 34 + lj + 1];
                         });
    }

    // FISTA from x_in (warm start) to x_out; returns updates made, sets gn
    __device__ int lower_solve(const T *b, const T *x_in, T *x_out, double eps, int max_iters,
                               double &gn, long long &passes)
    {
        const T *y = cx.y;
        compute_tau(b);
        for (long long i = gstart(); i < cx.N; i += gstride()) {
            const T v = __ldcg(x_in + i);
            cx.X0[i] = v;
            cx.X1[i] = v;
        }
        if (!sync()) return 0;
        T *x0 = cx.X0, *x1 = cx.X1, *x2 = cx.X2, *U = cx.U;
        double t = 1.0, theta = 0.0;
        int k = 0;
        const T al = (T)cx.alpha;
        T *sBl = sB;
        const double *tauc = tau;
        for (;; ++k) {
            const T th = (T)theta;
            // phase A: U = B y_k - y, y_k = x_k + theta (x_k - x_{k-1}) formed on the fly
            conv_pass(b, true,
                      [=](long long g) { const T a1 = __ldcg(x1 + g); return a1 + th * (a1 - __ldcg(x0 + g)); },
                      [](int, int, int, long long) {},
                      [=](int, int, int, long long g, T v) { U[g] = v - __ldg(y + g); return T(0); });
            if (!sync()) return k;
            // phase B: G = B^T U + alpha grad J(y_k); x_{k+1} = y_k - tau_c G; ||G||^2
            const double part = conv_pass(
                b, false, [=](long long g) { return __ldcg(U + g); },
                [=](int, int row0, int col0, long long cbase) {
                    load_tile(sBl, 34, cx.TH + 2, 34, cx.H, cx.W, cbase, row0 - 1, col0 - 1, [=](long long g) {
                        const T a1 = __ldcg(x1 + g);
                        return a1 + th * (a1 - __ldcg(x0 + g));
                    });
                },
                [=](int c, int li, int lj, long long g, T v) {
                    const T gr = v + al * tv_grad(sBl, li, lj);
                    x2[g] = sBl[(li + 1) * 34 + lj + 1] - (T)tauc[c] * gr;
                    return gr * gr;
                });
            const double ss = reduce(part, k & 1);
            if (!alive) return k;
            passes += 2;
            gn = sqrt(ss);
            if (!isfinite(gn)) { fail(ST_NONFINITE); return k; }
            if (gn <= eps || k >= max_iters) break;
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            theta = (t - 1.0) / tn;
            t = tn;
            T *tmp = x0; x0 = x1; x1 = x2; x2 = tmp;
        }
        const T th = (T)theta;
        for (long long i = gstart(); i < cx.N; i += gstride()) {
            const T a1 = __ldcg(x1 + i);
            x_out[i] = a1 + th * (a1 - __ldcg(x0 + i));
        }
        return k;
    }

    // r(b) = beta (w0 ||d||^2 + ||D_h d||^2 + ||D_v d||^2), d = b - a; every
    // CTA computes it (small); grad r into gr (may be null) by CTA 0's threads
    __device__ T dker(const T *b, long long idx) const { return __ldcg(b + idx) - __ldg(cx.a + idx); }

    __device__ double sobolev(const T *b)
    {
        const int K = cx.K, KK = K * K;
        double s = 0.0;
        for (int e = tid; e < cx.C * KK; e += NT) {
            const int c = e / KK, pq = e - c * KK, p = pq / K, q = pq - p * K;
            const long long base = (long long)c * KK;
            const double d = (double)dker(b, base + pq);
            const double dh = q < K - 1 ? (double)dker(b, base + pq + 1) - d : 0.0;
            const double dv = p < K - 1 ? (double)dker(b, base + pq + K) - d : 0.0;
            s += cx.w0 * d * d + dh * dh + dv * dv;
        }
        return cx.beta * block_sum(s, red);
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

    // ell = g(x) + r(b) and ||grad g(x)||; grad g stored in cx.G
    __device__ void upper_loss(const T *b, const T *x, double &loss, double &gxn, long long &passes)
    {
        const T *y = cx.y;
        T *V = cx.V, *G = cx.G;
        // r(b) first: b may be rewritten by other CTAs right after the last
        // barrier of this function (the next backtracking trial)
        const double rb = sobolev(b);
        const double pg = conv_pass(cx.a, true, [=](long long g) { return __ldcg(x + g); },
                                    [](int, int, int, long long) {},
                                    [=](int, int, int, long long g, T v) {
                                        const T e = v - __ldg(y + g);
                                        V[g] = e;
                                        return e * e;
                                    });
        const double gval = reduce(pg, 2);
        if (!alive) return;
        const double pgg = conv_pass(cx.a, false, [=](long long g) { return __ldcg(V + g); },
                                     [](int, int, int, long long) {},
                                     [=](int, int, int, long long g, T v) {
                                         const T gg = T(2) * v;
                                         G[g] = gg;
                                         return gg * gg;
                                     });
        const double ggs = reduce(pgg, 3);
        if (!alive) return;
        passes += 2;
        loss = gval + rb;
        gxn = sqrt(ggs);
        if (!isfinite(loss) || !isfinite(gxn)) fail(ST_NONFINITE);
    }

    // CG on H(x, b) q = rhs from the q held in Q (zero_start: Q is taken as
    // zero and cleared).  Returns iterations; sets res and capped.
    __device__ int cg(const T *b, const T *x, const T *rhs, T *Q, double delta, int max_iters,
                      bool zero_start, double &res, int &capped, long long &passes)
    {
        T *R = cx.R, *P = cx.P, *HP = cx.HP;
        double rrp = 0.0;
        if (zero_start) {
            for (long long i = gstart(); i < cx.N; i += gstride()) {
                const T v = __ldcg(rhs + i);
                Q[i] = T(0);
                R[i] = v;
                P[i] = v;
                rrp += (double)v * (double)v;
            }
        } else {
            hess_vec(b, x, Q, HP);
            if (!sync()) return 0;
            passes += 2;
            for (long long i = gstart(); i < cx.N; i += gstride()) {
                const T v = __ldcg(rhs + i) - __ldcg(HP + i);
                R[i] = v;
                P[i] = v;
                rrp += (double)v * (double)v;
            }
        }
        double rr = reduce(rrp, 4);
        if (!alive) return 0;
        int it = 0;
        capped = 0;
        while (sqrt(rr) > delta && it < max_iters) {
            const double php = reduce(hess_vec(b, x, P, HP), 5);
            if (!alive) return it;
            passes += 2;
            if (!isfinite(php)) { fail(ST_NONFINITE); return it; }
            if (!(php > 0.0)) { capped = 1; break; }
            const T a = (T)(rr / php);
            double rn = 0.0;
            for (long long i = gstart(); i < cx.N; i += gstride()) {
                const T pv = __ldcg(P + i);
                Q[i] = __ldcg(Q + i) + a * pv;
                const T rv = __ldcg(R + i) - a * __ldcg(HP + i);
                R[i] = rv;
                rn += (double)rv * (double)rv;
            }
            const double rr_new = reduce(rn, 6);
            if (!alive) return it;
            ++it;
            if (!isfinite(rr_new)) { fail(ST_NONFINITE); return it; }
            if (sqrt(rr_new) <= delta) { rr = rr_new; break; }
            const T be = (T)(rr_new / rr);
            rr = rr_new;
            for (long long i = gstart(); i < cx.N; i += gstride()) P[i] = __ldcg(R + i) + be * __ldcg(P + i);
            if (!sync()) return it;
        }
        res = sqrt(rr);
        if (res > delta) capped = 1;
        return it;
    }

    // out[c,p,q] = sum_ij x[c,i-p+r,j-q+r] (B v)[c,i,j] + v[c,i-p+r,j-q+r] (B x - y)[c,i,j];
    // z = -out (+ grad r(b) when add_r); written to zout; returns ||z||^2
    __device__ double cross(const T *b, const T *x, const T *v, T *zout, bool negate, bool add_r,
                            long long &passes)
    {
        const T *y = cx.y;
        T *U = cx.U, *V = cx.V;
        constexpr int MR = Cfg<T>::MR;
        const int r = cx.r, K = cx.K, KK = K * K, H = cx.H, W = cx.W;
        const int CKK = cx.C * KK;
        // phase K1: U = B v, V = B x - y
        for (int t = blockIdx.x; t < cx.ntiles; t += gridDim.x) {
            int c, row0, col0;
            tile_of(t, c, row0, col0);
            const long long cbase = (long long)c * cx.HW;
            load_w(b, c, true);
            load_tile(sA, pitch, cx.TH + 2 * r, 32 + 2 * r, H, W, cbase, row0 - r, col0 - r,
                      [=](long long g) { return __ldcg(v + g); });
            load_tile(sB, pitch, cx.TH + 2 * r, 32 + 2 * r, H, W, cbase, row0 - r, col0 - r,
                      [=](long long g) { return __ldcg(x + g); });
            __syncthreads();
            T au[MR], av[MR];
#pragma unroll
            for (int m = 0; m < MR; ++m) { au[m] = T(0); av[m] = T(0); }
            const int li0 = warp * MR;
            corr_strip<T, MR>(sA, pitch, sw, K, li0, lane, au);
            corr_strip<T, MR>(sB, pitch, sw, K, li0, lane, av);
            const int gj = col0 + lane;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int gi = row0 + li0 + m;
                if (gi < H && gj < W) {
                    const long long g = cbase + (long long)gi * W + gj;
                    U[g] = au[m];
                    V[g] = av[m] - __ldg(y + g);
                }
            }
            __syncthreads();
        }
        if (!sync()) return 0.0;
        // phase K2: per-CTA lag sums over its tiles
        double *zp = cx.zpart + (long long)blockIdx.x * CKK;
        for (int e = tid; e < CKK; e += NT) zp[e] = 0.0;
        for (int t = blockIdx.x; t < cx.ntiles; t += gridDim.x) {
            int c, row0, col0;
            tile_of(t, c, row0, col0);
            const long long cbase = (long long)c * cx.HW;
            load_tile(sA, pitch, cx.TH + 2 * r, 32 + 2 * r, H, W, cbase, row0 - r, col0 - r,
                      [=](long long g) { return __ldcg(x + g); });
            load_tile(sB, pitch, cx.TH + 2 * r, 32 + 2 * r, H, W, cbase, row0 - r, col0 - r,
                      [=](long long g) { return __ldcg(v + g); });
            for (int e = tid; e < cx.TH * 32; e += NT) {
                const int li = e >> 5, lj = e & 31;
                const int gi = row0 + li, gj = col0 + lj;
                const bool in = gi < H && gj < W;
                const long long g = cbase + (long long)gi * W + gj;
                sU[e] = in ? __ldcg(U + g) : T(0);
                sV[e] = in ? __ldcg(V + g) : T(0);
            }
            __syncthreads();
            for (int l = tid; l < KK; l += NT) {
                const int p = l / K, q = l - p * K;
                const int off = (2 * r - p) * pitch + (2 * r - q);
                double acc = 0.0;
                for (int li = 0; li < cx.TH; ++li) {
                    T s = T(0);
                    const T *xa = sA + off + li * pitch, *va = sB + off + li * pitch;
                    const T *ur = sU + li * 32, *vr = sV + li * 32;
#pragma unroll 8
                    for (int lj = 0; lj < 32; ++lj) s = fma(xa[lj], ur[lj], fma(va[lj], vr[lj], s));
                    acc += (double)s;
                }
                zp[c * KK + l] += acc;
            }
            __syncthreads();
        }
        if (!sync()) return 0.0;
        // phase K3: fixed-order sum over CTAs, sign, Sobolev term
        const long long gs = gstride();
        for (long long e = gstart(); e < CKK; e += gs) {
            double s = 0.0;
            for (int cta = 0; cta < (int)gridDim.x; ++cta) s += __ldcg(cx.zpart + (long long)cta * CKK + e);
            double zz = negate ? -s : s;
            if (add_r) zz += grad_sobolev_elem(b, (int)e);
            zout[e] = (T)zz;
        }
        passes += 4;   // B v, B x and the two lag correlations
        if (!sync()) return 0.0;
        double s = 0.0;
        for (int e = tid; e < CKK; e += NT) { const double zv = (double)__ldcg(zout + e); s += zv * zv; }
        return block_sum(s, red);
    }

    // ------------------------------------------------------------ MAID
    __device__ void maid(const Job<T> &jb)
    {
        MaidIn st = jb.maid;
        T *b = jb.bio, *x = (T *)jb.x, *q = jb.q;
        const int CKK = cx.C * cx.K * cx.K;
        long long passes = 0;
        int ll_iters = 0, cg_iters = 0, ll_capped = 0, cg_capped = 0, trials = 0, rounds = 0, accepted = 0;
        double loss = 0.0, gxn = 0.0, znorm = 0.0, psi = 0.0, gn = 0.0, res = 0.0;
        int j = st.max_bt;
        for (int round = 0; round < st.max_rounds && alive; ++round, ++j) {
            rounds = round + 1;
            // InexactGradient(b_k, eps_k, delta_k)
            ll_iters += lower_solve(b, x, x, st.eps, st.ll_max_iters, gn, passes);
            if (!sync()) break;
            if (gn > st.eps) ll_capped = 1;
            double l0 = 0.0, gx0 = 0.0;
            upper_loss(b, x, l0, gx0, passes);
            if (!alive) break;
            int capped = 0;
            cg_iters += cg(b, x, cx.G, q, st.delta, st.cg_max_iters, true, res, capped, passes);
            if (!alive) break;
            if (capped) cg_capped = 1;
            if (!sync()) break;
            const double zz = cross(b, x, q, cx.ZK, true, true, passes);
            if (!alive) break;
            znorm = sqrt(zz);
            if (!isfinite(znorm)) { fail(ST_NONFINITE); break; }
            bool done = false;
            for (int i = 0; i < j; ++i) {
                ++trials;
                // b' = b - step z (every CTA writes the same values to its share)
                for (long long e = gstart(); e < CKK; e += gstride())
                    cx.BT[e] = (T)((double)__ldcg(b + e) - st.step * (double)__ldcg(cx.ZK + e));
                if (!sync()) break;
                double g1 = 0.0;
                ll_iters += lower_solve(cx.BT, x, cx.XT, st.eps, st.ll_max_iters, g1, passes);
                if (!sync()) break;
                if (g1 > st.eps) ll_capped = 1;
                double l1 = 0.0, gx1 = 0.0;
                upper_loss(cx.BT, cx.XT, l1, gx1, passes);
                if (!alive) break;
                const double eb = st.eps;
                psi = l1 + gx1 * eb + 0.5 * st.L_gx * eb * eb - l0 + gx0 * eb + st.lambda * st.step * zz;
                if (psi <= 0.0) {
                    for (long long e = gstart(); e < CKK; e += gstride()) b[e] = __ldcg(cx.BT + e);
                    for (long long e = gstart(); e < cx.N; e += gstride()) x[e] = __ldcg(cx.XT + e);
                    loss = l1;
                    gxn = gx1;
                    st.eps *= st.nu_up;
                    st.delta *= st.nu_up;
                    st.step *= st.rho_up;
                    st.k += 1;
                    accepted = 1;
                    done = true;
                    break;
                }
                st.step *= st.rho_down;
            }
            if (done || !alive) break;
            loss = l0;
            gxn = gx0;
            st.eps *= st.nu_down;
            st.delta *= st.nu_down;
        }
        if (tid == 0 && blockIdx.x == 0) {
            DevOut *o = cx.out;
            o->accepted = accepted; o->rounds = rounds; o->trials = trials;
            o->ll_iters = ll_iters; o->cg_iters = cg_iters; o->ll_capped = ll_capped; o->cg_capped = cg_capped;
            o->k = st.k; o->eps = st.eps; o->delta = st.delta; o->step = st.step;
            o->loss = loss; o->gradx_norm = gxn; o->znorm = znorm; o->psi = psi;
            o->conv_passes = passes;
        }
    }
};

template <typename T>
__global__ void __launch_bounds__(NT) adp_kernel(const __grid_constant__ Ctx<T> cx,
                                                  const __grid_constant__ Job<T> jb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NW];
    __shared__ double bcast;
    __shared__ double tau[MAXC];
    __shared__ int sflag;
    Eng<T> e(cx, smem_raw, red, &bcast, tau, &sflag);
    const bool lead = threadIdx.x == 0 && blockIdx.x == 0;
    long long passes = 0;
    switch (jb.mode) {
    case M_APPLY_B: e.apply(jb.b, jb.x, jb.xo, false); break;
    case M_APPLY_BT: e.apply(jb.b, jb.x, jb.xo, true); break;
    case M_GRAD_LOWER: e.grad_lower(jb.b, jb.x, jb.xo); break;
    case M_HESS_VEC: e.hess_vec(jb.b, jb.x, jb.v, jb.xo); break;
    case M_LOWER_SOLVE: {
        double gn = 0.0;
        const int it = e.lower_solve(jb.b, jb.x, jb.xo, jb.eps, jb.max_iters, gn, passes);
        if (lead) { cx.out->iters = it; cx.out->gradnorm = gn; cx.out->capped = gn > jb.eps; cx.out->conv_passes = passes; }
        break;
    }
    case M_UPPER_LOSS: {
        double loss = 0.0, gxn = 0.0;
        e.upper_loss(jb.b, jb.x, loss, gxn, passes);
        if (e.alive && jb.xo) {
            for (long long i = e.gstart(); i < cx.N; i += e.gstride()) jb.xo[i] = __ldcg(cx.G + i);
        }
        if (lead) { cx.out->loss = loss; cx.out->gradx_norm = gxn; cx.out->conv_passes = passes; }
        break;
    }
    case M_HYPERGRAD: {
        const bool given = jb.v != nullptr;
        double gxn = 0.0, loss = 0.0;
        const T *rhs = jb.v;
        if (!given) {
            e.upper_loss(jb.b, jb.x, loss, gxn, passes);
            if (!e.alive) break;
            rhs = cx.G;
        }
        double res = 0.0;
        int capped = 0;
        const int it = e.cg(jb.b, jb.x, rhs, jb.q, jb.delta, jb.max_iters, false, res, capped, passes);
        if (!e.alive) break;
        if (!e.sync()) break;
        const double zz = e.cross(jb.b, jb.x, jb.q, jb.z, true, !given, passes);
        if (lead) {
            cx.out->cg_iters = it; cx.out->resnorm = res; cx.out->capped = capped;
            cx.out->znorm = sqrt(zz); cx.out->conv_passes = passes;
        }
        break;
    }
    case M_CROSS: e.cross(jb.b, jb.x, jb.v, jb.z, false, false, passes); break;
    case M_MAID: e.maid(jb); break;
    default: break;
    }
}

} // namespace adp
