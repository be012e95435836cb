// libadp: GB300 (sm_103a) hot path of ADP-beta solved by MAID (arXiv 2502.09758).
//
// One cooperative, persistent kernel per C-ABI call.  A call runs a program of
// phases (convolution passes over image strips, element-wise updates, FP64
// reductions) separated by a bounded grid barrier; the iteration control of
// FISTA (Algorithm 1, step 1), CG (Algorithm 1, step 2) and MAID (Algorithm 2)
// runs on the device, identically in every CTA, from reduction results that
// every CTA sums in the same order.  The host sees only the final scalars.
//
// This file is the host side: argument checks, workspace, cooperative launches.
// The kernels live in adp_engine.cuh, instantiated in adp_f32.cu / adp_f64.cu.
#include "adp_device.cuh"
#include "adp.h"

#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <type_traits>

using namespace adp;

namespace adp {
const void *kernel_f32();
const void *kernel_f64();
} // namespace adp

static thread_local char g_err[512];

namespace adp {
// lets the other translation units of the library report through adp_last_error
void record_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
} // namespace adp

static adp_status set_err(adp_status s, const char *fmt, const char *a = "", long long v = 0)
{
    snprintf(g_err, sizeof g_err, fmt, a, v);
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return set_err(ADP_ECUDA, "%s (code %lld)", cudaGetErrorString(e_), (long long)e_); \
    } while (0)

struct adp_problem {
    adp_params prm;
    cudaStream_t stream;
    int device, grid, nw;  // CTAs of the cooperative launch, warps per CTA
    size_t smem;           // dynamic shared memory per CTA (bytes)
    size_t esize;
    Geom g;                // padded layout and strips
    void *ws;              // NBUF padded images
    void *wg;              // two slots of both kernel orientations (global, read through L1)
    void *a;
    void *BT, *ZK;
    double *part, *zpart;
    unsigned *bar;
    DevOut *dout, *hout;
    double *a_host;        // a in FP64 on the host (for L of grad g)
    long long *trace;      // optional barrier trace (2 * trace_cap values)
    int trace_cap;
    CUtensorMap map_s, map_1, map_i;
    cudaEvent_t ev0, ev1;  // bracket the cooperative launch on the problem's stream
    float last_ms;
};

// ------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn(char *err, int errlen)
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
    });
    if (!fn) snprintf(err, errlen, "cuTensorMapEncodeTiled is not available from the driver");
    return fn;
}

namespace adp {
int encode_tensor_maps(void *ws, int nbuf, int C, const Geom &g, int esize, int MR, int NX, CUtensorMap *map_s,
                       CUtensorMap *map_1, CUtensorMap *map_i, char *err, int errlen)
{
    EncodeTiledFn fn = encode_fn(err, errlen);
    if (!fn) return 1;
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    // [buffer][channel][padded row][padded column], innermost first
    const cuuint64_t dims[4] = {(cuuint64_t)g.Wp, (cuuint64_t)g.Hp, (cuuint64_t)C, (cuuint64_t)nbuf};
    const cuuint64_t strides[3] = {(cuuint64_t)g.Wp * esize, (cuuint64_t)g.HWp * esize,
                                   (cuuint64_t)g.Np * esize};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const cuuint32_t box_s[4] = {(cuuint32_t)g.BW, (cuuint32_t)NX, 1, 1};
    const cuuint32_t box_1[4] = {40, (cuuint32_t)(MR + 2), 1, 1};
    const cuuint32_t box_i[4] = {32, (cuuint32_t)MR, 1, 1};
    struct { CUtensorMap *m; const cuuint32_t *box; const char *name; } maps[3] = {
        {map_s, box_s, "stage"}, {map_1, box_1, "halo-1"}, {map_i, box_i, "interior"}};
    for (auto &m : maps) {
        const CUresult r = fn(m.m, dt, 4, ws, dims, strides, m.box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(err, errlen, "tensor map encoding (%s box) failed with CUresult %d", m.name, (int)r);
            return 1;
        }
    }
    return 0;
}
} // namespace adp

template <typename T>
static Ctx<T> make_ctx(const adp_problem *p)
{
    Ctx<T> c;
    memset(&c, 0, sizeof c);
    const adp_params &q = p->prm;
    const Geom &g = p->g;
    c.map_s = p->map_s; c.map_1 = p->map_1; c.map_i = p->map_i;
    c.C = q.C; c.H = q.H; c.W = q.W; c.K = q.K; c.r = g.r; c.Kp = g.Kp;
    c.r4 = g.r4; c.Gx = g.Gx; c.Gy = g.Gy; c.Wp = g.Wp; c.Hp = g.Hp; c.BW = g.BW;
    c.nx = g.nx; c.ny = g.ny; c.nstrips = g.nstrips; c.wsm = g.wsm; c.multiwrap = g.multiwrap;
    c.N = g.N; c.HW = g.HW; c.HWp = g.HWp; c.Np = g.Np;
    c.trace = p->trace; c.trace_cap = p->trace_cap;
    c.reg = q.reg; c.alpha = q.alpha; c.rp = q.reg_param; c.beta = q.beta; c.w0 = q.sobolev_w0;
    c.ddphi_max = q.reg == ADP_REG_QUAD ? 1.0 : 1.0 / q.reg_param;
    c.alphaT = (T)q.alpha; c.rpT = (T)q.reg_param; c.irpT = (T)(1.0 / q.reg_param);
    c.ws = (T *)p->ws; c.wg = (T *)p->wg; c.a = (const T *)p->a;
    c.BT = (T *)p->BT; c.ZK = (T *)p->ZK;
    c.part = p->part; c.zpart = p->zpart; c.bar = p->bar; c.out = p->dout;
    const double to = q.wait_timeout_s > 0 ? q.wait_timeout_s : 2.0;
    c.timeout_ns = (long long)(to * 1e9);
    return c;
}

template <typename T>
static adp_status launch(adp_problem *p, Job<T> &jb)
{
    Ctx<T> cx = make_ctx<T>(p);
    CK(cudaSetDevice(p->device));
    CK(cudaMemsetAsync(p->bar, 0, sizeof(unsigned), p->stream));
    CK(cudaMemsetAsync(p->dout, 0, sizeof(DevOut), p->stream));
    void *args[] = {(void *)&cx, (void *)&jb};
    const void *fn = std::is_same<T, float>::value ? kernel_f32() : kernel_f64();
    CK(cudaEventRecord(p->ev0, p->stream));
    CK(cudaLaunchCooperativeKernel(fn, dim3(p->grid), dim3(32 * p->nw), args, p->smem, p->stream));
    CK(cudaEventRecord(p->ev1, p->stream));
    CK(cudaMemcpyAsync(p->hout, p->dout, sizeof(DevOut), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaEventElapsedTime(&p->last_ms, p->ev0, p->ev1));
    const int st = p->hout->status;
    if (st == ST_TIMEOUT) return set_err(ADP_ETIMEOUT, "device-side wait gave up after %s%lld ns", "", cx.timeout_ns);
    if (st == ST_NONFINITE) return set_err(ADP_ENONFINITE, "non-finite value in a reduction%s", "", 0);
    if (st != ST_OK) return set_err(ADP_ECUDA, "unexpected device status%s %lld", "", st);
    return ADP_OK;
}

static adp_status dispatch_job(adp_problem *p, int mode, const void *b, const void *x, void *xo, const void *v,
                               void *q, void *z, void *bio, double eps, double delta, int max_iters,
                               const MaidIn *mi)
{
    if (p->prm.prec == ADP_F32) {
        Job<float> j{};
        j.mode = mode; j.b = (const float *)b; j.x = (const float *)x; j.xo = (float *)xo;
        j.v = (const float *)v; j.q = (float *)q; j.z = (float *)z; j.bio = (float *)bio;
        j.eps = eps; j.delta = delta; j.max_iters = max_iters;
        if (mi) j.maid = *mi;
        return launch<float>(p, j);
    }
    Job<double> j{};
    j.mode = mode; j.b = (const double *)b; j.x = (const double *)x; j.xo = (double *)xo;
    j.v = (const double *)v; j.q = (double *)q; j.z = (double *)z; j.bio = (double *)bio;
    j.eps = eps; j.delta = delta; j.max_iters = max_iters;
    if (mi) j.maid = *mi;
    return launch<double>(p, j);
}

extern "C" {

const char *adp_last_error(void) { return g_err; }

const char *adp_status_string(adp_status s)
{
    switch (s) {
    case ADP_OK: return "ok";
    case ADP_EINVAL: return "invalid argument";
    case ADP_ENOMEM: return "out of device memory";
    case ADP_ECUDA: return "CUDA error";
    case ADP_ENONFINITE: return "non-finite value";
    case ADP_ENOCONV: return "iteration cap reached";
    case ADP_ELSFAIL: return "line search failed";
    case ADP_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

void adp_problem_destroy(adp_problem *p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->stream);
    void *ptrs[] = {p->ws, p->wg, p->a, p->BT, p->ZK, p->part, p->zpart, p->bar, p->dout, p->trace};
    for (void *q : ptrs) if (q) cudaFree(q);
    if (p->hout) cudaFreeHost(p->hout);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    free(p->a_host);
    free(p);
}

adp_status adp_problem_create(const adp_params *prm, const void *y, const void *a, void *stream,
                              adp_problem **out)
{
    if (!prm || !y || !a || !out) return set_err(ADP_EINVAL, "null argument%s", "", 0);
    *out = nullptr;
    const adp_params &q = *prm;
    if (q.C < 1 || q.C > MAXC) return set_err(ADP_EINVAL, "C must be in [1, 64]%s (got %lld)", "", q.C);
    if (q.H < 1 || q.W < 1) return set_err(ADP_EINVAL, "H and W must be positive%s", "", 0);
    if (q.K < 1 || q.K > KMAX || (q.K % 2) == 0)
        return set_err(ADP_EINVAL, "K must be odd and in [1, 63]%s (got %lld)", "", q.K);
    if (q.prec != ADP_F32 && q.prec != ADP_F64) return set_err(ADP_EINVAL, "unsupported precision%s", "", 0);
    if (q.reg < 0 || q.reg > 2) return set_err(ADP_EINVAL, "unknown regulariser%s", "", 0);
    if (q.reg != ADP_REG_QUAD && !(q.reg_param > 0)) return set_err(ADP_EINVAL, "reg_param must be > 0%s", "", 0);
    if (!(q.alpha >= 0) || !(q.beta >= 0)) return set_err(ADP_EINVAL, "alpha and beta must be >= 0%s", "", 0);

    adp_problem *p = (adp_problem *)calloc(1, sizeof(adp_problem));
    if (!p) return set_err(ADP_ENOMEM, "host allocation failed%s", "", 0);
    p->prm = q;
    p->stream = (cudaStream_t)stream;
    p->esize = q.prec == ADP_F32 ? sizeof(float) : sizeof(double);
    p->g = q.prec == ADP_F32 ? make_geom<float>(q.C, q.H, q.W, q.K) : make_geom<double>(q.C, q.H, q.W, q.K);
    const Geom &g = p->g;
    const int MR = q.prec == ADP_F32 ? Cfg<float>::MR : Cfg<double>::MR;
    const int NX = q.prec == ADP_F32 ? Cfg<float>::PC + MR - 1 : Cfg<double>::PC + MR - 1;

    adp_status st = ADP_OK;
#define CKC(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            st = set_err(e_ == cudaErrorMemoryAllocation ? ADP_ENOMEM : ADP_ECUDA, "%s (code %lld)", \
                         cudaGetErrorString(e_), (long long)e_);                             \
            adp_problem_destroy(p);                                                          \
            return st;                                                                       \
        }                                                                                    \
    } while (0)

    CKC(cudaGetDevice(&p->device));
    int nsm = 0, maxsmem = 0;
    CKC(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    CKC(cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    // warps per CTA: as many as shared memory allows (the kernel's static shared
    // memory is below 5 KB; keep that margin)
    int nw = MAXNW, total = 0;
    for (; nw >= 1; --nw) {
        total = q.prec == ADP_F32 ? Layout<float>(q.C, q.K, nw, g.wsm).total : Layout<double>(q.C, q.K, nw, g.wsm).total;
        if ((size_t)total * p->esize + 128 + 5 * 1024 <= (size_t)maxsmem) break;
    }
    if (nw < 1) {
        adp_problem_destroy(p);
        return set_err(ADP_EINVAL, "kernel too large for shared memory%s (K = %lld)", "", q.K);
    }
    p->nw = nw;
    p->smem = (size_t)total * p->esize + 128;   // + alignment slack of the TMA destinations
    const void *kfn = q.prec == ADP_F32 ? kernel_f32() : kernel_f64();
    // opt in to the device's whole dynamic shared memory (less the static part)
    // rather than this problem's size: the attribute is shared by every problem
    // on the device, and a smaller value set for a later problem with a smaller
    // K would make launches of an earlier, larger problem fail
    CKC(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem - 5 * 1024));
    int occ = 0;
    CKC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, 32 * nw, p->smem));
    if (occ < 1) {
        adp_problem_destroy(p);
        return set_err(ADP_EINVAL, "kernel cannot be resident%s", "", 0);
    }
    // grid: first spread the strips over the SMs (one CTA per SM, one strip per
    // warp); beyond that add CTAs up to the co-residency limit
    const long long maxgrid = (long long)occ * nsm;
    long long grid;
    if (g.nstrips <= (long long)nsm * nw) grid = g.nstrips < nsm ? g.nstrips : nsm;
    else grid = ((long long)g.nstrips + nw - 1) / nw;
    if (grid > maxgrid) grid = maxgrid;
    if (grid > GT_MAX) grid = GT_MAX;   // staging buffer of the grid totals
    p->grid = (int)grid;

    const size_t KK = (size_t)q.C * q.K * q.K;
    const size_t wsbytes = (size_t)NBUF * g.Np * p->esize;
    CKC(cudaMalloc(&p->ws, wsbytes));
    CKC(cudaMalloc(&p->wg, (size_t)4 * q.C * q.K * g.Kp * p->esize));
    CKC(cudaMalloc(&p->a, KK * p->esize));
    CKC(cudaMalloc(&p->BT, KK * p->esize));
    CKC(cudaMalloc(&p->ZK, KK * p->esize));
    CKC(cudaMalloc((void **)&p->part, (size_t)NSLOT * p->grid * sizeof(double)));
    CKC(cudaMalloc((void **)&p->zpart, (size_t)p->grid * p->nw * KK * sizeof(double)));
    CKC(cudaMalloc((void **)&p->bar, sizeof(unsigned)));
    CKC(cudaMalloc((void **)&p->dout, sizeof(DevOut)));
    CKC(cudaMallocHost((void **)&p->hout, sizeof(DevOut)));
    CKC(cudaEventCreate(&p->ev0));
    CKC(cudaEventCreate(&p->ev1));
    {
        char emsg[200];
        if (encode_tensor_maps(p->ws, NBUF, q.C, g, (int)p->esize, MR, NX, &p->map_s, &p->map_1, &p->map_i, emsg,
                               sizeof emsg)) {
            adp_problem_destroy(p);
            record_error(emsg);
            return ADP_ECUDA;
        }
    }
    CKC(cudaMemcpyAsync(p->a, a, KK * p->esize, cudaMemcpyDeviceToDevice, p->stream));
    CKC(cudaMemsetAsync(p->ws, 0, wsbytes, p->stream));
    p->a_host = (double *)malloc(KK * sizeof(double));
    if (!p->a_host) { adp_problem_destroy(p); return set_err(ADP_ENOMEM, "host allocation failed%s", "", 0); }
    if (q.prec == ADP_F32) {
        float *tmp = (float *)malloc(KK * sizeof(float));
        if (!tmp) { adp_problem_destroy(p); return set_err(ADP_ENOMEM, "host allocation failed%s", "", 0); }
        CKC(cudaMemcpyAsync(tmp, a, KK * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
        CKC(cudaStreamSynchronize(p->stream));
        for (size_t i = 0; i < KK; ++i) p->a_host[i] = tmp[i];
        free(tmp);
    } else {
        CKC(cudaMemcpyAsync(p->a_host, a, KK * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        CKC(cudaStreamSynchronize(p->stream));
    }
#undef CKC
    // y into its padded buffer (ghosts included); the caller may free y afterwards
    st = dispatch_job(p, M_IMPORT_Y, nullptr, y, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, nullptr);
    if (st != ADP_OK) {
        adp_problem_destroy(p);
        return st;
    }
    *out = p;
    return ADP_OK;
}

#define NEED(p, ...)                                                                  \
    do {                                                                              \
        if (!(p)) return set_err(ADP_EINVAL, "null problem%s", "", 0);                \
        const void *ptrs_[] = {__VA_ARGS__};                                          \
        for (const void *q_ : ptrs_)                                                  \
            if (!q_) return set_err(ADP_EINVAL, "null data pointer%s", "", 0);        \
    } while (0)

adp_status adp_apply_B(adp_problem *p, const void *b, const void *x, void *out)
{
    NEED(p, b, x, out);
    return dispatch_job(p, M_APPLY_B, b, x, out, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, nullptr);
}

adp_status adp_apply_Bt(adp_problem *p, const void *b, const void *z, void *out)
{
    NEED(p, b, z, out);
    return dispatch_job(p, M_APPLY_BT, b, z, out, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, nullptr);
}

adp_status adp_grad_lower(adp_problem *p, const void *b, const void *x, void *out, double *norm)
{
    NEED(p, b, x);
    adp_status s = dispatch_job(p, M_GRAD_LOWER, b, x, out, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, nullptr);
    if (s == ADP_OK && norm) *norm = p->hout->gradnorm;
    return s;
}

adp_status adp_hess_vec(adp_problem *p, const void *b, const void *x, const void *v, void *out)
{
    NEED(p, b, x, v, out);
    return dispatch_job(p, M_HESS_VEC, b, x, out, v, nullptr, nullptr, nullptr, 0, 0, 0, nullptr);
}

adp_status adp_lower_solve(adp_problem *p, const void *b, void *x, double eps, int max_iters, int *iters,
                           double *gradnorm)
{
    NEED(p, b, x);
    if (max_iters < 0) return set_err(ADP_EINVAL, "max_iters must be >= 0%s", "", 0);
    adp_status s = dispatch_job(p, M_LOWER_SOLVE, b, x, x, nullptr, nullptr, nullptr, nullptr, eps, 0, max_iters,
                                nullptr);
    if (s != ADP_OK) return s;
    if (iters) *iters = p->hout->iters;
    if (gradnorm) *gradnorm = p->hout->gradnorm;
    return p->hout->capped ? ADP_ENOCONV : ADP_OK;
}

adp_status adp_upper_loss(adp_problem *p, const void *b, const void *x, double *loss, double *gradx_norm,
                          void *gradx)
{
    NEED(p, b, x);
    adp_status s = dispatch_job(p, M_UPPER_LOSS, b, x, gradx, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, nullptr);
    if (s != ADP_OK) return s;
    if (loss) *loss = p->hout->loss;
    if (gradx_norm) *gradx_norm = p->hout->gradx_norm;
    return ADP_OK;
}

adp_status adp_hypergrad(adp_problem *p, const void *b, const void *x, const void *rhs, double delta,
                         int max_iters, void *q, void *z, int *cg_iters, double *resnorm)
{
    NEED(p, b, x, q, z);
    if (max_iters < 0) return set_err(ADP_EINVAL, "max_iters must be >= 0%s", "", 0);
    adp_status s = dispatch_job(p, M_HYPERGRAD, b, x, nullptr, rhs, q, z, nullptr, 0, delta, max_iters, nullptr);
    if (s != ADP_OK) return s;
    if (cg_iters) *cg_iters = p->hout->cg_iters;
    if (resnorm) *resnorm = p->hout->resnorm;
    return p->hout->capped ? ADP_ENOCONV : ADP_OK;
}

adp_status adp_cross_t(adp_problem *p, const void *b, const void *x, const void *v, void *out)
{
    NEED(p, b, x, v, out);
    return dispatch_job(p, M_CROSS, b, x, nullptr, v, nullptr, out, nullptr, 0, 0, 0, nullptr);
}

adp_status adp_maid_init(adp_problem *p, adp_maid_state *s)
{
    if (!p || !s) return set_err(ADP_EINVAL, "null argument%s", "", 0);
    memset(s, 0, sizeof *s);
    s->eps = 1e-2; s->delta = 1e-2; s->step = 0.1;
    s->lambda = 1e-4; s->rho_up = 1.1; s->rho_down = 0.5; s->nu_up = 1.25; s->nu_down = 0.5;
    s->max_bt = 5; s->max_rounds = 20; s->ll_max_iters = 300; s->cg_max_iters = 1000;
    const int K = p->prm.K;
    double m = 0.0;
    for (int c = 0; c < p->prm.C; ++c) {
        double l1 = 0.0;
        for (int e = 0; e < K * K; ++e) l1 += fabs(p->a_host[(size_t)c * K * K + e]);
        if (l1 * l1 > m) m = l1 * l1;
    }
    s->L_gx = 2.0 * m;
    return ADP_OK;
}

adp_status adp_maid_step(adp_problem *p, adp_maid_state *s, void *b, void *x, void *q)
{
    NEED(p, s, b, x, q);
    if (s->max_bt < 1 || s->max_rounds < 1 || s->ll_max_iters < 0 || s->cg_max_iters < 0)
        return set_err(ADP_EINVAL, "invalid MAID state%s", "", 0);
    MaidIn mi;
    mi.eps = s->eps; mi.delta = s->delta; mi.step = s->step; mi.lambda = s->lambda;
    mi.rho_up = s->rho_up; mi.rho_down = s->rho_down; mi.nu_up = s->nu_up; mi.nu_down = s->nu_down;
    mi.L_gx = s->L_gx; mi.eps_stop = s->eps_stop; mi.max_bt = s->max_bt; mi.max_rounds = s->max_rounds;
    mi.ll_max_iters = s->ll_max_iters; mi.cg_max_iters = s->cg_max_iters; mi.k = s->k;
    adp_status st = dispatch_job(p, M_MAID, nullptr, x, nullptr, nullptr, q, nullptr, b, 0, 0, 0, &mi);
    if (st != ADP_OK) return st;
    const DevOut *o = p->hout;
    s->eps = o->eps; s->delta = o->delta; s->step = o->step; s->k = o->k;
    s->accepted = o->accepted; s->rounds = o->rounds; s->trials = o->trials;
    s->ll_iters = o->ll_iters; s->cg_iters = o->cg_iters; s->ll_capped = o->ll_capped; s->cg_capped = o->cg_capped;
    s->loss = o->loss; s->gradx_norm = o->gradx_norm; s->znorm = o->znorm; s->psi = o->psi;
    s->stopped = o->stopped;
    return (o->accepted || o->stopped) ? ADP_OK : ADP_ELSFAIL;
}

adp_status adp_selftest_wait_timeout(adp_problem *p)
{
    if (!p) return set_err(ADP_EINVAL, "null problem%s", "", 0);
    if (p->grid < 2) return set_err(ADP_EINVAL, "the self-test needs a launch of at least 2 CTAs (this problem has %s%lld)", "", p->grid);
    return dispatch_job(p, M_WAIT_SELFTEST, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, 0,
                        nullptr);
}

long long adp_conv_passes_last(adp_problem *p) { return p ? p->hout->conv_passes : -1; }
int adp_grid_size(adp_problem *p) { return p ? p->grid : -1; }
int adp_warps_per_cta(adp_problem *p) { return p ? p->nw : -1; }
double adp_last_kernel_ms(adp_problem *p) { return p ? (double)p->last_ms : -1.0; }

adp_status adp_trace_enable(adp_problem *p, int cap)
{
    if (!p || cap < 0) return set_err(ADP_EINVAL, "invalid trace request%s", "", 0);
    CK(cudaSetDevice(p->device));
    CK(cudaStreamSynchronize(p->stream));
    if (p->trace) { CK(cudaFree(p->trace)); p->trace = nullptr; }
    p->trace_cap = 0;
    if (cap > 0) {
        cudaError_t e = cudaMalloc((void **)&p->trace, (size_t)2 * cap * sizeof(long long));
        if (e != cudaSuccess) return set_err(ADP_ENOMEM, "%s (code %lld)", cudaGetErrorString(e), (long long)e);
        CK(cudaMemsetAsync(p->trace, 0, (size_t)2 * cap * sizeof(long long), p->stream));
        p->trace_cap = cap;
    }
    return ADP_OK;
}

int adp_trace_read(adp_problem *p, long long *host_out, int cap)
{
    if (!p || !host_out || !p->trace) return -1;
    int n = p->hout->barriers < p->trace_cap ? p->hout->barriers : p->trace_cap;
    if (n > cap) n = cap;
    if (n > 0 && cudaMemcpy(host_out, p->trace, (size_t)2 * n * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    return n;
}

} // extern "C"
