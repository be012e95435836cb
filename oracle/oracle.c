/*
 * FP64 CPU oracle for ADP-beta solved by MAID (arXiv 2502.09758).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or helper with the CUDA
 * library; its own structs are declared here and mirrored in oracle/__init__.py.
 *
 * Style: plain loops in the order the paper states each step, double precision
 * everywhere, no blocking, no fusion, single thread.  Each function names the
 * passage it follows.
 *
 * Notation (Sec. 2, Eq. 2.4-2.5; Sec. 3.2):
 *   x       image, planar C x H x W, periodic boundary
 *   b, a    per-channel K x K kernels (b learned, a = kernel of A), r = (K-1)/2
 *   B x     (b * x)[c,i,j] = sum_{p,q} b[c,p,q] x[c, i-p+r, j-q+r]   (indices mod H, W)
 *   h(x,b)  = 1/2 ||B x - y||^2 + alpha J(x)            (lower level, Eq. 2.5b)
 *   g(x)    = ||A x - y||^2                              (upper fidelity, Sec. 3.2)
 *   r(b)    = beta (w0 ||b-a||^2 + ||D_h(b-a)||^2 + ||D_v(b-a)||^2)   (Sobolev, Sec. 4.2)
 *   J(x)    = sum phi((D_h x)) + phi((D_v x)), anisotropic, per channel
 *
 * Readings where the paper is silent or garbled (each one is listed with its
 * reason in the design notes): h carries the factor 1/2; the stopping test of
 * Algorithm 1 uses mu := 1; the step of the lower solver is 1/L_c with
 * L_c = ||b_c||_1^2 + 8 alpha max phi''; plain FISTA momentum; CG starts from
 * the given q; eps_bar = eps_k inside psi; L of grad_x ell = 2 max_c ||a_c||_1^2.
 *
 * Parity status: every function here is pinned by tests/test_oracle_pins.py
 * (closed forms, library routines, adjoint identities, finite differences,
 * Lemma 1 and Lemma 2).  The paper prints no numeric worked example, so the
 * paper's own figure values cannot be used as pins.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* regulariser kinds: smoothed TV variants and the quadratic case used by the
 * Fourier pins */
enum { ORC_REG_HUBER = 0, ORC_REG_SQRT = 1, ORC_REG_QUAD = 2 };

typedef struct {
    int C, H, W, K;
    double alpha;      /* lower-level weight of J            */
    double reg_param;  /* gamma (Huber) or nu (sqrt); unused for QUAD */
    int reg;           /* ORC_REG_*                           */
    double beta;       /* Sobolev weight of the upper level   */
    double w0;         /* weight of ||b-a||^2 in the H1 norm (1 full, 0 seminorm) */
} orc_prob;

typedef struct {
    /* adaptive quantities of Algorithm 2 */
    double eps, delta, step;
    /* hyper-parameters of Algorithm 2 and Eq. 3.4 */
    double lambda, rho_up, rho_down, nu_up, nu_down, L_gx;
    double eps_stop;       /* stop rule of Sec. 4.2: stop once eps <= eps_stop (0: off) */
    int max_bt, max_rounds, ll_max_iters, cg_max_iters;
    int k;                 /* upper iterations accepted so far */
    /* report of the last call */
    int accepted, rounds, trials, ll_iters, cg_iters, ll_capped, cg_capped, stopped;
    double loss, gradx_norm, znorm, psi;
} orc_maid;

static int wrap(int i, int n) { int m = i % n; return m < 0 ? m + n : m; }

static size_t nimg(const orc_prob *p) { return (size_t)p->C * p->H * p->W; }
static size_t nker(const orc_prob *p) { return (size_t)p->C * p->K * p->K; }

static double dot(const double *u, const double *v, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += u[i] * v[i];
    return s;
}

double orc_norm(const double *u, long n) { return sqrt(dot(u, u, (size_t)n)); }

/* ---------------------------------------------------------------- operators */

/* B x: the discrete integral operator T(b, x) of Eq. 2.4, a centred periodic
 * convolution per channel. */
void orc_conv(const orc_prob *p, const double *b, const double *x, double *out)
{
    int C = p->C, H = p->H, W = p->W, K = p->K, r = (K - 1) / 2;
    for (int c = 0; c < C; ++c)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double s = 0.0;
                for (int pp = 0; pp < K; ++pp)
                    for (int qq = 0; qq < K; ++qq)
                        s += b[((size_t)c * K + pp) * K + qq] *
                             x[((size_t)c * H + wrap(i - pp + r, H)) * W + wrap(j - qq + r, W)];
                out[((size_t)c * H + i) * W + j] = s;
            }
}

/* B^T z: the adjoint of orc_conv (a correlation with the same kernel), used in
 * the gradient of Prop. 1. */
void orc_conv_adj(const orc_prob *p, const double *b, const double *z, double *out)
{
    int C = p->C, H = p->H, W = p->W, K = p->K, r = (K - 1) / 2;
    for (int c = 0; c < C; ++c)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double s = 0.0;
                for (int pp = 0; pp < K; ++pp)
                    for (int qq = 0; qq < K; ++qq)
                        s += b[((size_t)c * K + pp) * K + qq] *
                             z[((size_t)c * H + wrap(i + pp - r, H)) * W + wrap(j + qq - r, W)];
                out[((size_t)c * H + i) * W + j] = s;
            }
}

/* Forward differences with periodic boundary (the discrete gradient of the TV
 * regulariser in Sec. 4.2) and their adjoints. */
void orc_dh(const orc_prob *p, const double *x, double *out)
{
    for (int c = 0; c < p->C; ++c)
        for (int i = 0; i < p->H; ++i)
            for (int j = 0; j < p->W; ++j) {
                size_t row = ((size_t)c * p->H + i) * p->W;
                out[row + j] = x[row + wrap(j + 1, p->W)] - x[row + j];
            }
}

void orc_dv(const orc_prob *p, const double *x, double *out)
{
    for (int c = 0; c < p->C; ++c)
        for (int i = 0; i < p->H; ++i)
            for (int j = 0; j < p->W; ++j)
                out[((size_t)c * p->H + i) * p->W + j] =
                    x[((size_t)c * p->H + wrap(i + 1, p->H)) * p->W + j] -
                    x[((size_t)c * p->H + i) * p->W + j];
}

void orc_dh_adj(const orc_prob *p, const double *w, double *out)
{
    for (int c = 0; c < p->C; ++c)
        for (int i = 0; i < p->H; ++i)
            for (int j = 0; j < p->W; ++j) {
                size_t row = ((size_t)c * p->H + i) * p->W;
                out[row + j] = w[row + wrap(j - 1, p->W)] - w[row + j];
            }
}

void orc_dv_adj(const orc_prob *p, const double *w, double *out)
{
    for (int c = 0; c < p->C; ++c)
        for (int i = 0; i < p->H; ++i)
            for (int j = 0; j < p->W; ++j)
                out[((size_t)c * p->H + i) * p->W + j] =
                    w[((size_t)c * p->H + wrap(i - 1, p->H)) * p->W + j] -
                    w[((size_t)c * p->H + i) * p->W + j];
}

/* ------------------------------------------------------------- regulariser */

/* phi and its derivatives.  Sqrt: the smoothed TV of Sec. 4.2,
 * phi(t) = sqrt(t^2 + nu^2) - nu.  Huber: t^2/(2 gamma) on |t| <= gamma, else
 * |t| - gamma/2 (tie in the quadratic branch).  Quad: t^2/2. */
double orc_phi(const orc_prob *p, double t)
{
    double g = p->reg_param;
    switch (p->reg) {
    case ORC_REG_HUBER: return fabs(t) <= g ? t * t / (2.0 * g) : fabs(t) - 0.5 * g;
    case ORC_REG_SQRT:  return sqrt(t * t + g * g) - g;
    default:            return 0.5 * t * t;
    }
}

double orc_dphi(const orc_prob *p, double t)
{
    double g = p->reg_param;
    switch (p->reg) {
    case ORC_REG_HUBER: return fabs(t) <= g ? t / g : (t > 0 ? 1.0 : -1.0);
    case ORC_REG_SQRT:  return t / sqrt(t * t + g * g);
    default:            return t;
    }
}

double orc_ddphi(const orc_prob *p, double t)
{
    double g = p->reg_param;
    switch (p->reg) {
    case ORC_REG_HUBER: return fabs(t) <= g ? 1.0 / g : 0.0;
    case ORC_REG_SQRT: { double s = t * t + g * g; return g * g / (s * sqrt(s)); }
    default:            return 1.0;
    }
}

/* sup phi'' (the constant C_J of Prop. 1 divided by ||D||^2) */
double orc_ddphi_max(const orc_prob *p)
{
    switch (p->reg) {
    case ORC_REG_HUBER: return 1.0 / p->reg_param;
    case ORC_REG_SQRT:  return 1.0 / p->reg_param;
    default:            return 1.0;
    }
}

double orc_J(const orc_prob *p, const double *x)
{
    size_t n = nimg(p);
    double *dh = malloc(n * sizeof *dh), *dv = malloc(n * sizeof *dv);
    orc_dh(p, x, dh);
    orc_dv(p, x, dv);
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += orc_phi(p, dh[i]) + orc_phi(p, dv[i]);
    free(dh); free(dv);
    return s;
}

/* grad J = D_h^T phi'(D_h x) + D_v^T phi'(D_v x) */
void orc_gradJ(const orc_prob *p, const double *x, double *out)
{
    size_t n = nimg(p);
    double *dh = malloc(n * sizeof *dh), *dv = malloc(n * sizeof *dv);
    double *t = malloc(n * sizeof *t);
    orc_dh(p, x, dh);
    orc_dv(p, x, dv);
    for (size_t i = 0; i < n; ++i) { dh[i] = orc_dphi(p, dh[i]); dv[i] = orc_dphi(p, dv[i]); }
    orc_dh_adj(p, dh, out);
    orc_dv_adj(p, dv, t);
    for (size_t i = 0; i < n; ++i) out[i] += t[i];
    free(dh); free(dv); free(t);
}

/* Hessian of J applied to v: D^T (phi''(D x) . D v) */
void orc_hessJ_vec(const orc_prob *p, const double *x, const double *v, double *out)
{
    size_t n = nimg(p);
    double *dh = malloc(n * sizeof *dh), *dv = malloc(n * sizeof *dv);
    double *vh = malloc(n * sizeof *vh), *vv = malloc(n * sizeof *vv);
    double *t = malloc(n * sizeof *t);
    orc_dh(p, x, dh); orc_dv(p, x, dv);
    orc_dh(p, v, vh); orc_dv(p, v, vv);
    for (size_t i = 0; i < n; ++i) {
        vh[i] *= orc_ddphi(p, dh[i]);
        vv[i] *= orc_ddphi(p, dv[i]);
    }
    orc_dh_adj(p, vh, out);
    orc_dv_adj(p, vv, t);
    for (size_t i = 0; i < n; ++i) out[i] += t[i];
    free(dh); free(dv); free(vh); free(vv); free(t);
}

/* ------------------------------------------------------------- lower level */

/* h(x, b) = 1/2 ||B x - y||^2 + alpha J(x)   (Eq. 2.5b, with the factor 1/2) */
double orc_h(const orc_prob *p, const double *b, const double *x, const double *y)
{
    size_t n = nimg(p);
    double *u = malloc(n * sizeof *u);
    orc_conv(p, b, x, u);
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += (u[i] - y[i]) * (u[i] - y[i]);
    free(u);
    return 0.5 * s + p->alpha * orc_J(p, x);
}

/* grad_x h = B^T (B x - y) + alpha grad J   (Prop. 1, gradient formula) */
void orc_grad_h(const orc_prob *p, const double *b, const double *x, const double *y, double *out)
{
    size_t n = nimg(p);
    double *u = malloc(n * sizeof *u), *t = malloc(n * sizeof *t);
    orc_conv(p, b, x, u);
    for (size_t i = 0; i < n; ++i) u[i] -= y[i];
    orc_conv_adj(p, b, u, out);
    orc_gradJ(p, x, t);
    for (size_t i = 0; i < n; ++i) out[i] += p->alpha * t[i];
    free(u); free(t);
}

/* grad^2_x h v = B^T B v + alpha D^T(phi''(D x) . D v)   (Prop. 1, Hessian) */
void orc_hess_h_vec(const orc_prob *p, const double *b, const double *x, const double *v, double *out)
{
    size_t n = nimg(p);
    double *u = malloc(n * sizeof *u), *t = malloc(n * sizeof *t);
    orc_conv(p, b, v, u);
    orc_conv_adj(p, b, u, out);
    orc_hessJ_vec(p, x, v, t);
    for (size_t i = 0; i < n; ++i) out[i] += p->alpha * t[i];
    free(u); free(t);
}

/* ------------------------------------------------- single outputs (sampling)
 * The same definitions evaluated at one pixel, for checks at image sizes where
 * the whole-image functions above would take too long.  Each restates its
 * whole-image counterpart at one output index. */

/* (B x)[c,i,j], Eq. 2.4 */
double orc_conv_at(const orc_prob *p, const double *b, const double *x, int c, int i, int j)
{
    int H = p->H, W = p->W, K = p->K, r = (K - 1) / 2;
    double s = 0.0;
    for (int pp = 0; pp < K; ++pp)
        for (int qq = 0; qq < K; ++qq)
            s += b[((size_t)c * K + pp) * K + qq] *
                 x[((size_t)c * H + wrap(i - pp + r, H)) * W + wrap(j - qq + r, W)];
    return s;
}

/* (B^T z)[c,i,j] */
double orc_conv_adj_at(const orc_prob *p, const double *b, const double *z, int c, int i, int j)
{
    int H = p->H, W = p->W, K = p->K, r = (K - 1) / 2;
    double s = 0.0;
    for (int pp = 0; pp < K; ++pp)
        for (int qq = 0; qq < K; ++qq)
            s += b[((size_t)c * K + pp) * K + qq] *
                 z[((size_t)c * H + wrap(i + pp - r, H)) * W + wrap(j + qq - r, W)];
    return s;
}

/* value of image u at (c, i, j) with periodic indices */
static double at(const orc_prob *p, const double *u, int c, int i, int j)
{
    return u[((size_t)c * p->H + wrap(i, p->H)) * p->W + wrap(j, p->W)];
}

/* (grad J)[c,i,j] = phi'(x_ij - x_i,j-1) - phi'(x_i,j+1 - x_ij)
 *                 + phi'(x_ij - x_i-1,j) - phi'(x_i+1,j - x_ij),
 * the entry of D_h^T phi'(D_h x) + D_v^T phi'(D_v x) at one pixel */
static double gradJ_at(const orc_prob *p, const double *x, int c, int i, int j)
{
    double xc = at(p, x, c, i, j);
    return orc_dphi(p, xc - at(p, x, c, i, j - 1)) - orc_dphi(p, at(p, x, c, i, j + 1) - xc) +
           orc_dphi(p, xc - at(p, x, c, i - 1, j)) - orc_dphi(p, at(p, x, c, i + 1, j) - xc);
}

/* (grad_x h)[c,i,j] = (B^T (B x - y))[c,i,j] + alpha (grad J)[c,i,j]; the
 * residual B x - y is formed at each of the K^2 pixels the adjoint reads */
double orc_grad_h_at(const orc_prob *p, const double *b, const double *x, const double *y, int c, int i, int j)
{
    int K = p->K, r = (K - 1) / 2;
    double s = 0.0;
    for (int pp = 0; pp < K; ++pp)
        for (int qq = 0; qq < K; ++qq) {
            int ii = wrap(i + pp - r, p->H), jj = wrap(j + qq - r, p->W);
            double u = orc_conv_at(p, b, x, c, ii, jj) - at(p, y, c, ii, jj);
            s += b[((size_t)c * K + pp) * K + qq] * u;
        }
    return s + p->alpha * gradJ_at(p, x, c, i, j);
}

/* (grad^2_x h v)[c,i,j] = (B^T B v)[c,i,j] + alpha (D^T(phi''(D x) . D v))[c,i,j] */
double orc_hess_h_vec_at(const orc_prob *p, const double *b, const double *x, const double *v, int c, int i,
                         int j)
{
    int K = p->K, r = (K - 1) / 2;
    double s = 0.0;
    for (int pp = 0; pp < K; ++pp)
        for (int qq = 0; qq < K; ++qq) {
            int ii = wrap(i + pp - r, p->H), jj = wrap(j + qq - r, p->W);
            s += b[((size_t)c * K + pp) * K + qq] * orc_conv_at(p, b, v, c, ii, jj);
        }
    double xc = at(p, x, c, i, j), vc = at(p, v, c, i, j);
    double hJ = orc_ddphi(p, xc - at(p, x, c, i, j - 1)) * (vc - at(p, v, c, i, j - 1)) -
                orc_ddphi(p, at(p, x, c, i, j + 1) - xc) * (at(p, v, c, i, j + 1) - vc) +
                orc_ddphi(p, xc - at(p, x, c, i - 1, j)) * (vc - at(p, v, c, i - 1, j)) -
                orc_ddphi(p, at(p, x, c, i + 1, j) - xc) * (at(p, v, c, i + 1, j) - vc);
    return s + p->alpha * hJ;
}

/* Lipschitz constant of grad_x h on channel c: ||B_c||^2 <= ||b_c||_1^2
 * (Young), plus alpha ||D||^2 sup phi'' with ||D||^2 = 8 in 2D. */
double orc_lipschitz(const orc_prob *p, const double *b, int c)
{
    double s = 0.0;
    for (int k = 0; k < p->K * p->K; ++k) s += fabs(b[(size_t)c * p->K * p->K + k]);
    return s * s + 8.0 * p->alpha * orc_ddphi_max(p);
}

/* Lower-level solve of Algorithm 1, first step: FISTA from the warm start x,
 * stopped as soon as ||grad_x h(y_k)|| <= eps (returning y_k) or after
 * max_iters updates.  Returns the number of updates. */
int orc_fista(const orc_prob *p, const double *b, const double *y, double *x,
              double eps, int max_iters, double *gradnorm)
{
    size_t n = nimg(p), hw = (size_t)p->H * p->W;
    double *xk = malloc(n * sizeof *xk), *yk = malloc(n * sizeof *yk);
    double *xn = malloc(n * sizeof *xn), *G = malloc(n * sizeof *G);
    double *tau = malloc((size_t)p->C * sizeof *tau);
    for (int c = 0; c < p->C; ++c) tau[c] = 1.0 / orc_lipschitz(p, b, c);
    memcpy(xk, x, n * sizeof *x);
    memcpy(yk, x, n * sizeof *x);
    double t = 1.0;
    int k = 0;
    for (;; ++k) {
        orc_grad_h(p, b, yk, y, G);
        double gn = orc_norm(G, (long)n);
        if (gn <= eps || k >= max_iters) { *gradnorm = gn; break; }
        for (size_t i = 0; i < n; ++i) xn[i] = yk[i] - tau[i / hw] * G[i];
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double theta = (t - 1.0) / tn;
        for (size_t i = 0; i < n; ++i) yk[i] = xn[i] + theta * (xn[i] - xk[i]);
        memcpy(xk, xn, n * sizeof *xn);
        t = tn;
    }
    memcpy(x, yk, n * sizeof *x);
    free(xk); free(yk); free(xn); free(G); free(tau);
    return k;
}

/* Algorithm 1, second step: conjugate gradients on grad^2_x h(x, b) q = rhs,
 * starting from the q given, stopped at ||residual|| <= delta or max_iters.
 * Returns the number of iterations; *capped is set when the tolerance was not
 * met (cap reached, or a non-positive curvature p^T H p). */
int orc_cg(const orc_prob *p, const double *b, const double *x, const double *rhs,
           double delta, int max_iters, double *q, double *resnorm, int *capped)
{
    size_t n = nimg(p);
    double *r = malloc(n * sizeof *r), *d = malloc(n * sizeof *d), *Hd = malloc(n * sizeof *Hd);
    orc_hess_h_vec(p, b, x, q, Hd);
    for (size_t i = 0; i < n; ++i) r[i] = rhs[i] - Hd[i];
    memcpy(d, r, n * sizeof *r);
    double rr = dot(r, r, n);
    int it = 0, bad = 0;
    while (sqrt(rr) > delta && it < max_iters) {
        orc_hess_h_vec(p, b, x, d, Hd);
        double dHd = dot(d, Hd, n);
        if (!(dHd > 0.0)) { bad = 1; break; }
        double a = rr / dHd;
        for (size_t i = 0; i < n; ++i) { q[i] += a * d[i]; r[i] -= a * Hd[i]; }
        double rr_new = dot(r, r, n);
        ++it;
        if (sqrt(rr_new) <= delta) { rr = rr_new; break; }
        double beta = rr_new / rr;
        for (size_t i = 0; i < n; ++i) d[i] = r[i] + beta * d[i];
        rr = rr_new;
    }
    *resnorm = sqrt(rr);
    *capped = bad || sqrt(rr) > delta;
    free(r); free(d); free(Hd);
    return it;
}

/* (grad^2_{xb} h(x, b))^T q, Algorithm 1 third step.  From
 * <grad_x h(x,b), q> = <B x - y, B q> + alpha <grad J(x), q>, the derivative in
 * b[c,p,q] is <S_pq x, B q> + <B x - y, S_pq q>, where (S_pq v)[i,j] =
 * v[i-p+r, j-q+r] is the image that b[c,p,q] multiplies inside B. */
void orc_cross_t(const orc_prob *p, const double *b, const double *x, const double *y,
                 const double *q, double *out)
{
    int C = p->C, H = p->H, W = p->W, K = p->K, r = (K - 1) / 2;
    size_t n = nimg(p);
    double *u = malloc(n * sizeof *u), *v = malloc(n * sizeof *v);
    orc_conv(p, b, q, u);                 /* u = B q         */
    orc_conv(p, b, x, v);                 /* v = B x - y     */
    for (size_t i = 0; i < n; ++i) v[i] -= y[i];
    for (int c = 0; c < C; ++c)
        for (int pp = 0; pp < K; ++pp)
            for (int qq = 0; qq < K; ++qq) {
                double s = 0.0;
                for (int i = 0; i < H; ++i)
                    for (int j = 0; j < W; ++j) {
                        size_t o = ((size_t)c * H + i) * W + j;
                        size_t sh = ((size_t)c * H + wrap(i - pp + r, H)) * W + wrap(j - qq + r, W);
                        s += x[sh] * u[o] + q[sh] * v[o];
                    }
                out[((size_t)c * K + pp) * K + qq] = s;
            }
    free(u); free(v);
}

/* ------------------------------------------------------------- upper level */

/* g(x) = ||A x - y||^2 (Sec. 3.2, no factor 1/2); grad g = 2 A^T (A x - y). */
double orc_g(const orc_prob *p, const double *a, const double *x, const double *y, double *grad)
{
    size_t n = nimg(p);
    double *e = malloc(n * sizeof *e);
    orc_conv(p, a, x, e);
    for (size_t i = 0; i < n; ++i) e[i] -= y[i];
    double g = dot(e, e, n);
    if (grad) {
        orc_conv_adj(p, a, e, grad);
        for (size_t i = 0; i < n; ++i) grad[i] *= 2.0;
    }
    free(e);
    return g;
}

/* Kernel forward differences inside the K x K array, Neumann (the last
 * difference is zero), used by the Sobolev penalty of Sec. 4.2. */
static void kdiff(int K, const double *d, double *dh, double *dv)
{
    for (int pp = 0; pp < K; ++pp)
        for (int qq = 0; qq < K; ++qq) {
            dh[pp * K + qq] = qq < K - 1 ? d[pp * K + qq + 1] - d[pp * K + qq] : 0.0;
            dv[pp * K + qq] = pp < K - 1 ? d[(pp + 1) * K + qq] - d[pp * K + qq] : 0.0;
        }
}

/* r(b) = beta (w0 ||d||^2 + ||D_h d||^2 + ||D_v d||^2), d = b - a; with grad
 * 2 beta (w0 d + D_h^T D_h d + D_v^T D_v d). */
double orc_r(const orc_prob *p, const double *b, const double *a, double *grad)
{
    int K = p->K;
    double *d = malloc((size_t)K * K * sizeof *d);
    double *dh = malloc((size_t)K * K * sizeof *dh), *dv = malloc((size_t)K * K * sizeof *dv);
    double s = 0.0;
    for (int c = 0; c < p->C; ++c) {
        const double *bc = b + (size_t)c * K * K, *ac = a + (size_t)c * K * K;
        for (int k = 0; k < K * K; ++k) d[k] = bc[k] - ac[k];
        kdiff(K, d, dh, dv);
        for (int k = 0; k < K * K; ++k) s += p->w0 * d[k] * d[k] + dh[k] * dh[k] + dv[k] * dv[k];
        if (grad) {
            double *gc = grad + (size_t)c * K * K;
            for (int pp = 0; pp < K; ++pp)
                for (int qq = 0; qq < K; ++qq) {
                    /* D^T w at (pp,qq) = w(before) - w(here), with zero outside
                     * the range where the difference is defined */
                    double th = (qq >= 1 ? dh[pp * K + qq - 1] : 0.0) - dh[pp * K + qq];
                    double tv = (pp >= 1 ? dv[(pp - 1) * K + qq] : 0.0) - dv[pp * K + qq];
                    gc[pp * K + qq] = 2.0 * p->beta * (p->w0 * d[pp * K + qq] + th + tv);
                }
        }
    }
    free(d); free(dh); free(dv);
    return p->beta * s;
}

/* Upper-level loss ell(x, b) = g(x) + r(b) and ||grad_x ell|| = ||grad g(x)||,
 * the ingredients of Eq. 3.4. */
double orc_upper(const orc_prob *p, const double *a, const double *b, const double *x,
                 const double *y, double *gradx_norm)
{
    size_t n = nimg(p);
    double *gg = malloc(n * sizeof *gg);
    double l = orc_g(p, a, x, y, gg) + orc_r(p, b, a, NULL);
    *gradx_norm = orc_norm(gg, (long)n);
    free(gg);
    return l;
}

/* Algorithm 1 steps 2-3: q from CG on grad^2_x h q = rhs (rhs = grad g(x) when
 * rhs is NULL) and z = -(grad^2_{xb} h)^T q + grad r(b); when an explicit rhs
 * is given (adjoint of an arbitrary upstream gradient) grad r is left out.
 * Returns CG iterations. */
int orc_hypergrad(const orc_prob *p, const double *a, const double *b, const double *x,
                  const double *y, const double *rhs, double delta, int cg_max,
                  double *q, double *z, double *resnorm, int *capped)
{
    size_t n = nimg(p), nk = nker(p);
    double *g = malloc(n * sizeof *g), *gr = calloc(nk, sizeof *gr);
    if (rhs) memcpy(g, rhs, n * sizeof *g);
    else orc_g(p, a, x, y, g);
    int it = orc_cg(p, b, x, g, delta, cg_max, q, resnorm, capped);
    orc_cross_t(p, b, x, y, q, z);
    if (!rhs) orc_r(p, b, a, gr);
    for (size_t k = 0; k < nk; ++k) z[k] = -z[k] + gr[k];
    free(g); free(gr);
    return it;
}

/* Defaults of Sec. 4.1 (eps0 = 1e-2, rho = 1.1 / 0.5, nu = 1.25 / 0.5,
 * alpha0 = 0.1, LL cap 300) and the readings lambda = 1e-4, max_BT = 5. */
void orc_maid_init(orc_maid *s)
{
    memset(s, 0, sizeof *s);
    s->eps = 1e-2; s->delta = 1e-2; s->step = 0.1;
    s->lambda = 1e-4; s->rho_up = 1.1; s->rho_down = 0.5; s->nu_up = 1.25; s->nu_down = 0.5;
    s->L_gx = 0.0;
    s->max_bt = 5; s->max_rounds = 20; s->ll_max_iters = 300; s->cg_max_iters = 1000;
}

/* One upper iteration k of Algorithm 2 (MAID) with the inexact sufficient
 * decrease psi of Eq. 3.4.  x holds x~(b_k) on entry (warm start) and
 * x~(b_{k+1}) on exit; q receives the last CG solution.  Returns 1 when a step
 * was accepted, 0 when the backtracking rounds ran out (b unchanged, eps/delta
 * and the step already shrunk).  The stop rule of Sec. 4.2 (the upper
 * iterations end once the accuracy eps reaches eps_stop) is checked on entry
 * and after every decrease of eps; when it fires the call returns 0 with
 * stopped = 1 and b unchanged. */
int orc_maid_step(const orc_prob *p, orc_maid *s, const double *a, const double *y,
                  double *b, double *x, double *q)
{
    size_t n = nimg(p), nk = nker(p);
    double *z = malloc(nk * sizeof *z), *bt = malloc(nk * sizeof *bt);
    double *xt = malloc(n * sizeof *xt);
    double gn, res;
    int capped, j = s->max_bt;
    s->accepted = 0; s->rounds = 0; s->trials = 0; s->ll_iters = 0; s->cg_iters = 0;
    s->ll_capped = 0; s->cg_capped = 0; s->stopped = 0;
    if (s->eps_stop > 0.0 && s->eps <= s->eps_stop) {
        s->stopped = 1;
        free(z); free(bt); free(xt);
        return 0;
    }
    for (int round = 0; round < s->max_rounds; ++round, ++j) {
        s->rounds = round + 1;
        /* InexactGradient(b_k, eps_k, delta_k) */
        int it = orc_fista(p, b, y, x, s->eps, s->ll_max_iters, &gn);
        s->ll_iters += it;
        if (gn > s->eps) s->ll_capped = 1;
        double gx0;
        double l0 = orc_upper(p, a, b, x, y, &gx0);
        memset(q, 0, n * sizeof *q);
        s->cg_iters += orc_hypergrad(p, a, b, x, y, NULL, s->delta, s->cg_max_iters, q, z, &res, &capped);
        if (capped) s->cg_capped = 1;
        double zz = dot(z, z, nk);
        s->znorm = sqrt(zz);
        for (int i = 0; i < j; ++i) {
            s->trials += 1;
            for (size_t k = 0; k < nk; ++k) bt[k] = b[k] - s->step * z[k];
            memcpy(xt, x, n * sizeof *x);
            s->ll_iters += orc_fista(p, bt, y, xt, s->eps, s->ll_max_iters, &gn);
            if (gn > s->eps) s->ll_capped = 1;
            double gx1;
            double l1 = orc_upper(p, a, bt, xt, y, &gx1);
            double eb = s->eps;   /* eps_bar_{k+1} = max(eps_k, eps_{k+1}) = eps_k */
            double psi = l1 + gx1 * eb + 0.5 * s->L_gx * eb * eb - l0 + gx0 * eb
                       + s->lambda * s->step * zz;
            s->psi = psi;
            if (psi <= 0.0) {
                memcpy(b, bt, nk * sizeof *b);
                memcpy(x, xt, n * sizeof *x);
                s->loss = l1; s->gradx_norm = gx1;
                s->eps *= s->nu_up; s->delta *= s->nu_up; s->step *= s->rho_up;
                s->k += 1;
                s->accepted = 1;
                free(z); free(bt); free(xt);
                return 1;
            }
            s->step *= s->rho_down;
        }
        s->loss = l0; s->gradx_norm = gx0;
        s->eps *= s->nu_down; s->delta *= s->nu_down;
        if (s->eps_stop > 0.0 && s->eps <= s->eps_stop) { s->stopped = 1; break; }
    }
    free(z); free(bt); free(xt);
    return 0;
}

/* L of grad_x ell = grad g in Eq. 3.4: 2 ||A||^2 <= 2 max_c ||a_c||_1^2. */
double orc_L_gx(const orc_prob *p, const double *a)
{
    double m = 0.0;
    for (int c = 0; c < p->C; ++c) {
        double s = 0.0;
        for (int k = 0; k < p->K * p->K; ++k) s += fabs(a[(size_t)c * p->K * p->K + k]);
        if (s * s > m) m = s * s;
    }
    return 2.0 * m;
}
