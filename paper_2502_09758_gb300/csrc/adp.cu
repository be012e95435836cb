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
#include "adp_tc.cuh"
#include "adp.h"

#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

using namespace adp;

namespace adp {
const void *kernel_f32();
const void *kernel_f64();
const void *kernel_f32_batched();
const void *kernel_f32_fft();
const void *kernel_f64_batched();
} // namespace adp

static thread_local char g_err[512];

namespace adp {
// lets the other translation units of the library report through adp_last_error
void record_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

// Opts kernel fn in to all the dynamic shared memory its static part leaves
// (the attribute is shared by every problem on the device, so it is the
// device maximum rather than one problem's size).
cudaError_t optin_dynamic_smem(const void *fn, int maxsmem)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem - (int)fa.sharedSizeBytes);
}
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
    size_t smem_fft;       // the same for the FFT-path kernel (adp_set_fft)
    int nw_fft;            // warps per CTA of the FFT-path kernel
    int grid_fft;          // CTAs of its cooperative launch
    int part_cap;          // CTAs the reduction slots (part) hold
    size_t zpart_cap;      // warps the per-warp kernel-gradient rows (zpart) hold
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
    CUtensorMap map_fz;     // FFT path: the half spectra fzh as a 2-D FP32 tensor
    cudaEvent_t ev0, ev1;  // bracket the cooperative launch on the problem's stream
    float last_ms;
    TcPlan *tc;            // BF16 tensor-core operator workspace (made on first use)
    TcTimes tc_times;
    // FFT operator path (adp_set_fft): on/off, log2 sizes, column block, buffers
    int fft, flogH, flogW, fcb, frb;
    float2 *fz, *fs, *fy, *ftw;  // complex scratch, kernel spectrum, second spectrum, twiddles (H/2, W/2)
    float *fout, *fc;       // correlation of the last FFT pass; B^T y of the current lower solve
    // real-to-complex pipeline of the FFT-path lower solve (fr2c = 0: not used)
    int fr2c, frp, fcb2, fpsh, fnst, fncs, fstage, fcstage, frows;
    float2 *fzh, *fzn;      // half spectra (C x H x W/2) and the column W/2 (C x H)
    float *fsh, *fsn;       // |F(k)|^2 at those columns
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

namespace adp {
int encode_bf16_swizzled_3d(void *base, const unsigned long long dims[3], const unsigned long long strides[2],
                            const unsigned box[3], CUtensorMap *map, char *err, int errlen)
{
    EncodeTiledFn fn = encode_fn(err, errlen);
    if (!fn) return 1;
    const cuuint64_t d[3] = {dims[0], dims[1], dims[2]};
    const cuuint64_t st[2] = {strides[0], strides[1]};
    const cuuint32_t bx[3] = {box[0], box[1], box[2]};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, d, st, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(err, errlen, "tensor map encoding (BF16 image) failed with CUresult %d", (int)r);
        return 1;
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
    c.map_s = p->map_s; c.map_1 = p->map_1; c.map_i = p->map_i; c.map_fz = p->map_fz;
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
    if (p->fft) {
        c.fft = 1; c.flogH = p->flogH; c.flogW = p->flogW; c.fcb = p->fcb; c.frb = p->frb;
        c.fz = p->fz; c.fs = p->fs; c.fy = p->fy; c.fout = (T *)p->fout; c.fc = (T *)p->fc;
        c.ftwH = p->ftw; c.ftwW = p->ftw + q.H / 2;
        c.fr2c = p->fr2c; c.frp = p->frp; c.fcb2 = p->fcb2; c.fpsh = p->fpsh; c.fnst = p->fnst;
        c.fstage = p->fstage; c.fcstage = p->fcstage; c.frows = p->frows; c.fncs = p->fncs;
        c.fzh = p->fzh; c.fzn = p->fzn; c.fsh = p->fsh; c.fsn = p->fsn;
    }
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
    const void *fn = std::is_same<T, float>::value ? (p->fft ? kernel_f32_fft() : kernel_f32()) : kernel_f64();
    CK(cudaEventRecord(p->ev0, p->stream));
    const bool fftk = std::is_same<T, float>::value && p->fft;
    CK(cudaLaunchCooperativeKernel(fn, dim3(fftk ? p->grid_fft : p->grid), dim3(32 * (fftk ? p->nw_fft : p->nw)),
                                   args, fftk ? p->smem_fft : p->smem, p->stream));
    CK(cudaEventRecord(p->ev1, p->stream));
    CK(cudaMemcpyAsync(p->hout, p->dout, sizeof(DevOut), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaEventElapsedTime(&p->last_ms, p->ev0, p->ev1));
    const int st = p->hout->status;
    if (st == ST_TIMEOUT) return set_err(ADP_ETIMEOUT, "device-side wait gave up after %s%lld ns", "", cx.timeout_ns);
    if (st == ST_NONFINITE) return set_err(ADP_ENONFINITE, "non-finite value in a reduction%s", "", 0);
    if (st == ST_ALIGN) return set_err(ADP_ECUDA, "dynamic shared memory not 128-byte aligned%s", "", 0);
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
    tc_plan_destroy(p->tc);
    void *fptrs[] = {p->fz, p->fs, p->fy, p->ftw, p->fout, p->fc, p->fzh, p->fzn, p->fsh, p->fsn};
    for (void *q : fptrs) if (q) cudaFree(q);
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
    if (g.Np >= (1LL << 31)) {     // pixel offsets inside a padded image are 32-bit
        adp_problem_destroy(p);
        return set_err(ADP_EINVAL, "padded image too large%s (%lld elements, limit 2^31)", "", g.Np);
    }
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
    for (; nw >= 2; nw -= 2) {   // warps work in pairs
        total = q.prec == ADP_F32 ? Layout<float>(q.C, q.K, nw, g.wsm).total : Layout<double>(q.C, q.K, nw, g.wsm).total;
        if ((size_t)total * p->esize + SMEM_STATIC_MARGIN <= (size_t)maxsmem) break;
    }
    if (nw < 2) {
        adp_problem_destroy(p);
        return set_err(ADP_EINVAL, "kernel too large for shared memory%s (K = %lld)", "", q.K);
    }
    p->nw = nw;
    p->smem = (size_t)total * p->esize;
    const void *kfn = q.prec == ADP_F32 ? kernel_f32() : kernel_f64();
    // opt in to the device's whole dynamic shared memory (less the static part)
    // rather than this problem's size: the attribute is shared by every problem
    // on the device, and a smaller value set for a later problem with a smaller
    // K would make launches of an earlier, larger problem fail
    CKC(optin_dynamic_smem(kfn, maxsmem));
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
    p->part_cap = p->grid;
    CKC(cudaMalloc((void **)&p->zpart, (size_t)p->grid * p->nw * KK * sizeof(double)));
    p->zpart_cap = (size_t)p->grid * p->nw;
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

static adp_status apply_bf16(adp_problem *p, const void *b, const void *x, void *out, bool transpose)
{
    NEED(p, b, x, out);
    if (p->prm.prec != ADP_F32) return set_err(ADP_EINVAL, "BF16 operator needs an ADP_F32 problem%s", "", 0);
    if (p->prm.K > TC_KMAX) return set_err(ADP_EINVAL, "BF16 operator supports K <= 33%s (K = %lld)", "", p->prm.K);
    CK(cudaSetDevice(p->device));
    char emsg[256];
    if (!p->tc) {
        const int rc = tc_plan_create(p->prm.C, p->prm.H, p->prm.W, p->prm.K, p->device, &p->tc, emsg, sizeof emsg);
        if (rc) {
            record_error(emsg);
            return rc == 1 ? ADP_EINVAL : rc == 2 ? ADP_ENOMEM : ADP_ECUDA;
        }
    }
    int dst = ST_OK;
    const long long timeout_ns = (long long)((p->prm.wait_timeout_s > 0 ? p->prm.wait_timeout_s : 2.0) * 1e9);
    if (tc_apply(p->tc, (const float *)b, (const float *)x, (float *)out, transpose, timeout_ns, p->stream,
                 &p->tc_times, &dst, emsg, sizeof emsg)) {
        record_error(emsg);
        return ADP_ECUDA;
    }
    p->last_ms = p->tc_times.corr_ms;
    if (dst == ST_TIMEOUT) return set_err(ADP_ETIMEOUT, "device-side wait gave up%s", "", 0);
    if (dst != ST_OK) return set_err(ADP_ECUDA, "unexpected device status%s %lld", "", dst);
    return ADP_OK;
}

adp_status adp_apply_B_bf16(adp_problem *p, const void *b, const void *x, void *out)
{
    return apply_bf16(p, b, x, out, false);
}

adp_status adp_apply_Bt_bf16(adp_problem *p, const void *b, const void *z, void *out)
{
    return apply_bf16(p, b, z, out, true);
}

static int log2_exact(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
}

adp_status adp_set_fft(adp_problem *p, int enable)
{
    if (!p) return set_err(ADP_EINVAL, "null problem%s", "", 0);
    if (!enable) {
        p->fft = 0;
        return ADP_OK;
    }
    const adp_params &q = p->prm;
    if (q.prec != ADP_F32) return set_err(ADP_EINVAL, "FFT path needs an ADP_F32 problem%s", "", 0);
    const int lh = log2_exact(q.H), lw = log2_exact(q.W);
    if (lh < 1 || lw < 1 || q.H > 8192 || q.W > 8192)
        return set_err(ADP_EINVAL, "FFT path needs H and W powers of two in 2..8192%s", "", 0);
    // the FFT-path kernel: FFT_WARPS warps per CTA, whose warp regions hold
    // only the epilogue tiles, up to FFT_CTAS_PER_SM CTAs per SM (so that
    // independent tasks overlap one another's latency): a grid of that many
    // CTAs per SM when the problem's own grid fills the SMs, else the
    // problem's grid; all the dynamic shared memory a co-resident CTA may have
    // (less the weights) is the scratch of the FFT phases
    const size_t esz = sizeof(float);
    const int nwf = FFT_WARPS;
    const Layout<float> L(q.C, q.K, nwf, p->g.wsm, true);
    CK(cudaSetDevice(p->device));
    size_t smem_fft = 0;
    int grid_fft = p->grid;
    {
        int nsm = 0, maxsmem = 0, occ = 0;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
        CK(cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
        CK(optin_dynamic_smem(kernel_f32_fft(), maxsmem));
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, kernel_f32_fft()));
        if (p->grid >= nsm) grid_fft = std::min(FFT_CTAS_PER_SM * nsm, GT_MAX);
        // the largest shared memory at which that grid stays co-resident
        for (size_t cand = (size_t)maxsmem - fa.sharedSizeBytes; cand >= (size_t)L.total * esz; cand -= 4096) {
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel_f32_fft(), 32 * nwf, cand));
            if ((long long)occ * nsm >= grid_fft) { smem_fft = cand; break; }
            if (cand < 4096 + (size_t)L.total * esz) break;
        }
        if (!smem_fft)
            return set_err(ADP_EINVAL, "FFT path: kernel not co-resident at its grid%s (%lld CTAs)", "", grid_fft);
    }
    if (grid_fft > p->part_cap) {      // reduction slots for the larger grid (kept once grown)
        double *np_ = nullptr;
        CK(cudaMalloc((void **)&np_, (size_t)NSLOT * grid_fft * sizeof(double)));
        CK(cudaFree(p->part));
        p->part = np_;
        p->part_cap = grid_fft;
    }
    const size_t scratch = smem_fft - (size_t)L.w_elems * esz;
    if ((size_t)q.W * 8 > scratch)
        return set_err(ADP_EINVAL, "FFT path: image rows too long for shared memory%s (W = %lld)", "", q.W);
    // columns per column block and rows per row batch: powers of two, at most
    // 32, within the scratch, and small enough that every CTA gets a block
    auto pick = [&](int len, int count_total, int limit) {
        int v = 32;
        while (v > 1 && ((size_t)len * v * 8 > scratch || v > limit || (long long)count_total / v < grid_fft)) v >>= 1;
        return v;
    };
    const int cb = pick(q.H, q.C * q.W, q.W), rb = pick(q.W, q.C * q.H, q.H);
    if ((size_t)q.H * cb * 8 > scratch)
        return set_err(ADP_EINVAL, "FFT path: image columns too long for shared memory%s (H = %lld)", "", q.H);
    const size_t scratch_r2c = scratch;
    if (!p->fz) {
        const size_t n = (size_t)q.C * q.H * q.W;
        CK(cudaMalloc((void **)&p->fz, n * sizeof(float2)));
        CK(cudaMalloc((void **)&p->fs, n * sizeof(float2)));
        CK(cudaMalloc((void **)&p->fy, n * sizeof(float2)));
        CK(cudaMalloc((void **)&p->fout, n * sizeof(float)));
        CK(cudaMalloc((void **)&p->fc, n * sizeof(float)));
        CK(cudaMalloc((void **)&p->ftw, (size_t)(q.H / 2 + q.W / 2) * sizeof(float2)));
        // twiddles exp(-2 pi i j / n), j < n/2, computed in double and rounded once
        std::vector<float2> tw((size_t)(q.H / 2 + q.W / 2));
        const double pi = 3.14159265358979323846;
        for (int j = 0; j < q.H / 2; ++j)
            tw[j] = make_float2((float)cos(2 * pi * j / q.H), (float)-sin(2 * pi * j / q.H));
        for (int j = 0; j < q.W / 2; ++j)
            tw[q.H / 2 + j] = make_float2((float)cos(2 * pi * j / q.W), (float)-sin(2 * pi * j / q.W));
        CK(cudaMemcpy(p->ftw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    p->flogH = lh;
    p->flogW = lw;
    p->fcb = cb;
    p->frb = rb;
    p->smem_fft = smem_fft;
    p->nw_fft = nwf;
    p->grid_fft = grid_fft;
    // the real-to-complex pipeline of the lower solve: row tasks of frp row
    // pairs (a radix-8 group for each thread where the image allows, and no
    // fewer tasks than CTAs), column tasks of fcb2 half-spectrum columns, double
    // buffered when both fit in the scratch (else single), padding of the
    // row transforms' slots against the bit-reversed reads; W >= 4 so that
    // every staged row is whole 16-byte copies
    p->fr2c = 0;
    if (q.W >= 4 && enable != 2) {
        // shared memory of a row task with rp row pairs: its half spectra
        // double buffered (2 rp rows of W/2 + 2 (W/64) float2 each), one buffer
        // of 6 rp + 2 image rows (FISTA: y with its halo, x, B^T y; the
        // Hessian product: p and x with their halos), the work area; of a
        // column task: two stages of its spectrum and of its symbol
        const size_t spp = (size_t)(q.W / 2) + 2 * (size_t)(q.W / 64);
        const int W2 = q.W / 2;
        int best_rp = 0, cb2 = 0, nst = 0, ncs = 0;
        size_t st_spc = 0, st_rows = 0;
        int ps = 31;
        for (int ns = 2; ns >= 1 && !best_rp; --ns)
            for (int rp = 1; rp <= q.H / 2; rp *= 2) {
                // no fewer tasks than CTAs, no more radix-8 groups than threads
                if (rp > 1 && ((long long)q.C * q.H / (2 * rp) < grid_fft || rp * q.W > 8 * 32 * nwf)) break;
                int lrp = 0;
                while ((1 << lrp) < rp) ++lrp;
                const int psr = lw + lrp >= 9 ? lw + lrp - 5 : 31;
                const size_t spc = 4 * (size_t)rp * spp, rows = (size_t)(6 * rp + 2) * q.W;     // floats
                const size_t work = ((size_t)rp * q.W + (((size_t)rp * q.W) >> psr) + 1) * 8;  // bytes
                if ((ns * spc + rows) * 4 + work > scratch) break;
                best_rp = rp;
                nst = ns;
                st_spc = spc;
                st_rows = rows;
                ps = psr;
            }
        for (int ns = 2; ns >= 1 && best_rp && !cb2; --ns)
            for (int c2 = W2 < 16 ? W2 : 16; c2 >= 2; c2 >>= 1) {
                // float2 spectrum + float symbol, stages rounded to 128 bytes (TMA destinations)
                if ((size_t)ns * (((size_t)q.H * c2 + 15) / 16 * 16) * 12 > scratch) continue;
                if (c2 > 2 && (long long)q.C * (W2 / c2) < grid_fft) continue;
                cb2 = c2;
                ncs = ns;
                break;
            }
        if (best_rp && cb2) {
            p->frp = best_rp;
            p->fpsh = ps;
            p->fnst = nst;
            p->fncs = ncs;
            p->fstage = (int)st_spc;
            p->frows = (int)st_rows;
            p->fcstage = (q.H * cb2 + 15) / 16 * 16;
            p->fcb2 = cb2;
            if (!p->fzh) {
                const size_t nh = (size_t)q.C * q.H * W2, nn = (size_t)q.C * q.H;
                CK(cudaMalloc((void **)&p->fzh, nh * sizeof(float2)));
                CK(cudaMalloc((void **)&p->fzn, nn * sizeof(float2)));
                CK(cudaMalloc((void **)&p->fsh, nh * sizeof(float)));
                CK(cudaMalloc((void **)&p->fsn, nn * sizeof(float)));
            }
            // fzh as FP32 [C*H][W]: a column task's block is the box of
            // 2 fcb2 floats x min(H, 256) rows, H / that many boxes per task
            {
                char emsg[160];
                EncodeTiledFn fn = encode_fn(emsg, sizeof emsg);
                if (!fn) return set_err(ADP_ECUDA, "%s", emsg);
                const cuuint64_t dims[2] = {(cuuint64_t)q.W, (cuuint64_t)q.C * q.H};
                const cuuint64_t strides[1] = {(cuuint64_t)W2 * sizeof(float2)};
                const cuuint32_t box[2] = {(cuuint32_t)(2 * cb2), (cuuint32_t)(q.H < 256 ? q.H : 256)};
                const cuuint32_t estr[2] = {1, 1};
                const CUresult r = fn(&p->map_fz, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->fzh, dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS)
                    return set_err(ADP_ECUDA, "tensor map encoding (half spectra) failed%s with CUresult %lld", "",
                                   (long long)r);
            }
            p->fr2c = 1;
        }
    }
    p->fft = 1;
    return ADP_OK;
}

int adp_fft_enabled(adp_problem *p) { return p ? p->fft : 0; }

adp_status adp_set_launch(adp_problem *p, int grid, int nw)
{
    if (!p) return set_err(ADP_EINVAL, "null problem%s", "", 0);
    const adp_params &q = p->prm;
    const Geom &g = p->g;
    if (nw < 2 || nw > MAXNW || (nw & 1)) return set_err(ADP_EINVAL, "warps per CTA must be even, 2..%s%lld", "", MAXNW);
    if (grid < 1 || grid > GT_MAX) return set_err(ADP_EINVAL, "grid must be 1..%s%lld CTAs", "", GT_MAX);
    CK(cudaSetDevice(p->device));
    int nsm = 0, maxsmem = 0, occ = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    CK(cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    const int total = q.prec == ADP_F32 ? Layout<float>(q.C, q.K, nw, g.wsm).total : Layout<double>(q.C, q.K, nw, g.wsm).total;
    const size_t smem = (size_t)total * p->esize;
    if (smem + SMEM_STATIC_MARGIN > (size_t)maxsmem)
        return set_err(ADP_EINVAL, "launch shape: warps' stages exceed shared memory%s (%lld warps)", "", nw);
    const void *kfn = q.prec == ADP_F32 ? kernel_f32() : kernel_f64();
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, 32 * nw, smem));
    if ((long long)occ * nsm < grid)
        return set_err(ADP_EINVAL, "launch shape: grid not co-resident%s (%lld CTAs)", "", grid);
    const size_t KK = (size_t)q.C * q.K * q.K;
    if (grid > p->part_cap) {
        double *np_ = nullptr;
        CK(cudaMalloc((void **)&np_, (size_t)NSLOT * grid * sizeof(double)));
        CK(cudaFree(p->part));
        p->part = np_;
        p->part_cap = grid;
    }
    if ((size_t)grid * nw > p->zpart_cap) {
        double *nz = nullptr;
        CK(cudaMalloc((void **)&nz, (size_t)grid * nw * KK * sizeof(double)));
        CK(cudaFree(p->zpart));
        p->zpart = nz;
        p->zpart_cap = (size_t)grid * nw;
    }
    p->grid = grid;
    p->nw = nw;
    p->smem = smem;
    return ADP_OK;
}

int adp_fft_pipeline(adp_problem *p) { return !p || !p->fft ? 0 : (p->fr2c ? 2 : 1); }

double adp_bf16_prep_ms_last(adp_problem *p) { return p && p->tc ? (double)p->tc_times.prep_ms : -1.0; }
int adp_bf16_grid_size(adp_problem *p) { return p ? tc_grid(p->tc) : 0; }

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
    mi.ll_max_iters = s->ll_max_iters; mi.cg_max_iters = s->cg_max_iters; mi.k = s->k; mi.halted = 0;
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

// ------------------------------------------------------------ batched MAID
struct adp_batch {
    std::vector<adp_problem *> ps;
    int n, prec, nw;
    size_t esize, ctx_bytes, job_bytes, smem;
    int max_ctas;              // co-resident CTAs of the batched kernel
    std::vector<int> first;    // group g = CTAs first[g] .. first[g+1]-1
    std::vector<double> work;  // balancer: estimated CTA-time of each problem's step
    void *dctx, *djob;         // launch records (device), n each
    int *dfirst;
    unsigned *dbar;            // one barrier counter per problem (256-byte stride)
    DevOut *dout, *hout;       // one result record per problem
    MaidTotals *dtot;          // running totals (graph runs)
    unsigned char *hctx, *hjob;   // pinned staging of the launch records
    cudaEvent_t ev0, ev1;
    float last_ms;
    cudaStream_t cs;              // capture / replay stream of device-resident runs
    cudaGraphExec_t gexec;        // instantiated graph of the last run shape
    int gsteps, ggrid;            // its steps and CTAs
    std::vector<unsigned char> gctx;   // batch of one: the records the graph captured by value
};

static const size_t kBarStride = 64;   // unsigned counters, 256 bytes apart

static void batch_free(adp_batch *bt)
{
    if (!bt) return;
    void *dev[] = {bt->dctx, bt->djob, bt->dfirst, bt->dbar, bt->dout, bt->dtot};
    for (void *q : dev) if (q) cudaFree(q);
    if (bt->hout) cudaFreeHost(bt->hout);
    if (bt->hctx) cudaFreeHost(bt->hctx);
    if (bt->hjob) cudaFreeHost(bt->hjob);
    if (bt->ev0) cudaEventDestroy(bt->ev0);
    if (bt->ev1) cudaEventDestroy(bt->ev1);
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    if (bt->cs) cudaStreamDestroy(bt->cs);
    delete bt;
}

// group sizes proportional to the work estimates, at least one CTA each and at
// most the problem's own grid (its reduction and gradient buffers are sized
// for that), summing to at most max_ctas
static void batch_partition(adp_batch *bt)
{
    const int n = bt->n;
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += bt->work[i];
    std::vector<int> g(n);
    int sum = 0;
    for (int i = 0; i < n; ++i) {
        int gi = (int)(bt->max_ctas * bt->work[i] / tot);
        gi = std::max(1, std::min(gi, bt->ps[i]->grid));
        g[i] = gi;
        sum += gi;
    }
    // hand out the remainder to the problems with the most work per CTA
    while (sum < bt->max_ctas) {
        int best = -1;
        double bw = 0.0;
        for (int i = 0; i < n; ++i)
            if (g[i] < bt->ps[i]->grid && bt->work[i] / g[i] > bw) { bw = bt->work[i] / g[i]; best = i; }
        if (best < 0) break;
        ++g[best];
        ++sum;
    }
    while (sum > bt->max_ctas) {   // only when rounding overshot: take from the least loaded
        int best = -1;
        double bw = 1e300;
        for (int i = 0; i < n; ++i)
            if (g[i] > 1 && bt->work[i] / g[i] < bw) { bw = bt->work[i] / g[i]; best = i; }
        if (best < 0) break;
        --g[best];
        --sum;
    }
    bt->first.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) bt->first[i + 1] = bt->first[i] + g[i];
}

template <typename T>
static void batch_fill(adp_batch *bt, const adp_maid_state *st, void *const *b, void *const *x, void *const *q,
                       bool resident, int max_steps)
{
    for (int i = 0; i < bt->n; ++i) {
        adp_problem *p = bt->ps[i];
        Ctx<T> c = make_ctx<T>(p);
        c.bar = bt->dbar + i * kBarStride;
        c.out = bt->dout + i;
        c.totals = resident ? bt->dtot + i : nullptr;
        c.trace = nullptr;
        // a batch of several problems runs the direct operator (the FFT scratch
        // is sized for a problem's own launch shape, which only a batch of one keeps)
        if (bt->n > 1) c.fft = 0;
        c.trace_cap = 0;
        memcpy(bt->hctx + i * bt->ctx_bytes, &c, sizeof c);
        Job<T> j;
        memset(&j, 0, sizeof j);
        j.mode = M_MAID;
        j.x = (const T *)x[i];
        j.q = (T *)q[i];
        j.bio = (T *)b[i];
        const adp_maid_state *s = st + i;
        MaidIn &mi = j.maid;
        mi.eps = s->eps; mi.delta = s->delta; mi.step = s->step; mi.lambda = s->lambda;
        mi.rho_up = s->rho_up; mi.rho_down = s->rho_down; mi.nu_up = s->nu_up; mi.nu_down = s->nu_down;
        mi.L_gx = s->L_gx; mi.eps_stop = s->eps_stop; mi.max_bt = s->max_bt; mi.max_rounds = s->max_rounds;
        mi.ll_max_iters = s->ll_max_iters; mi.cg_max_iters = s->cg_max_iters; mi.k = s->k; mi.halted = 0;
        j.maid_home = resident ? (MaidIn *)((unsigned char *)bt->djob + i * bt->job_bytes + offsetof(Job<T>, maid))
                               : nullptr;
        j.max_steps = resident ? max_steps : 0;
        memcpy(bt->hjob + i * bt->job_bytes, &j, sizeof j);
    }
}

// records of problem i after a launch: report into st[i] (and the state, from
// the result record or, for device-resident runs, from the job's MAID state)
static adp_status batch_report(adp_batch *bt, adp_maid_state *st, const MaidIn *resident_state)
{
    adp_status first_bad = ADP_OK;
    for (int i = 0; i < bt->n; ++i) {
        const DevOut *o = bt->hout + i;
        adp_maid_state *s = st + i;
        if (o->status == ST_TIMEOUT && first_bad == ADP_OK) first_bad = set_err(ADP_ETIMEOUT, "device-side wait gave up%s", "", 0);
        if (o->status == ST_NONFINITE && first_bad == ADP_OK) first_bad = set_err(ADP_ENONFINITE, "non-finite value in a reduction%s", "", 0);
        if (o->status != ST_OK && first_bad == ADP_OK)
            first_bad = set_err(ADP_ECUDA, "unexpected device status for problem %s%lld", "", i);
        if (o->status != ST_OK) continue;
        if (resident_state) {
            const MaidIn &m = resident_state[i];
            s->eps = m.eps; s->delta = m.delta; s->step = m.step; s->k = m.k;
        } else if (o->rounds > 0 || o->stopped) {
            s->eps = o->eps; s->delta = o->delta; s->step = o->step; s->k = o->k;
        }
        s->accepted = o->accepted; s->rounds = o->rounds; s->trials = o->trials;
        s->ll_iters = o->ll_iters; s->cg_iters = o->cg_iters; s->ll_capped = o->ll_capped; s->cg_capped = o->cg_capped;
        s->loss = o->loss; s->gradx_norm = o->gradx_norm; s->znorm = o->znorm; s->psi = o->psi;
        s->stopped = o->stopped;
        if (!resident_state && !o->accepted && !o->stopped && first_bad == ADP_OK)
            first_bad = set_err(ADP_ELSFAIL, "MAID backtracking rounds exhausted for problem %s%lld", "", i);
    }
    return first_bad;
}

// balancer: a group's CTA-time (device time x CTAs) estimates its work for the
// next launch; half the old estimate, half the measurement (both normalised)
static void batch_rebalance(adp_batch *bt)
{
    bool any = false;
    std::vector<double> w(bt->n);
    for (int i = 0; i < bt->n; ++i) {
        const double t = (double)(bt->hout[i].t_end - bt->hout[i].t_start);
        const int gsz = bt->first[i + 1] - bt->first[i];
        w[i] = t > 0 ? t * gsz : 0.0;
        if (w[i] > 0) any = true;
    }
    if (any) {
        double mn = 1e300, sw = 0.0, so = 0.0;
        for (int i = 0; i < bt->n; ++i) if (w[i] > 0) mn = std::min(mn, w[i]);
        for (int i = 0; i < bt->n; ++i) {
            if (w[i] <= 0) w[i] = mn;
            sw += w[i];
            so += bt->work[i];
        }
        for (int i = 0; i < bt->n; ++i) bt->work[i] = 0.5 * bt->work[i] / so + 0.5 * w[i] / sw;
        batch_partition(bt);
    }
}

// One batched launch.  A batch of one problem launches the single-problem
// kernel with its records by value (parameter space, as adp_maid_step does);
// a device-resident run then finds its MAID state through the job's maid_home.
static adp_status batch_launch(adp_batch *bt, cudaStream_t stream)
{
    const bool one = bt->n == 1;
    const void *fn = one ? (bt->prec == ADP_F32 ? (bt->ps[0]->fft ? kernel_f32_fft() : kernel_f32()) : kernel_f64())
                         : (bt->prec == ADP_F32 ? kernel_f32_batched() : kernel_f64_batched());
    void *ctxp = bt->dctx, *jobp = bt->djob;
    int *fp = bt->dfirst;
    int n = bt->n;
    void *args_many[] = {&ctxp, &jobp, &fp, &n};
    void *args_one[] = {bt->hctx, bt->hjob};
    void **args = one ? args_one : args_many;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    const bool fftk = one && bt->prec == ADP_F32 && bt->ps[0]->fft;
    cfg.gridDim = dim3((unsigned)(fftk ? bt->ps[0]->grid_fft : bt->first[n]));
    cfg.blockDim = dim3(32 * (fftk ? bt->ps[0]->nw_fft : bt->nw));
    cfg.dynamicSmemBytes = fftk ? bt->ps[0]->smem_fft : bt->smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    CK(cudaMemsetAsync(bt->dbar, 0, (size_t)bt->n * kBarStride * sizeof(unsigned), stream));
    CK(cudaMemsetAsync(bt->dout, 0, (size_t)bt->n * sizeof(DevOut), stream));
    CK(cudaLaunchKernelExC(&cfg, fn, args));
    return ADP_OK;
}

extern "C" {

adp_status adp_batch_create(adp_problem *const *ps, int n, adp_batch **out)
{
    if (!ps || !out || n < 1) return set_err(ADP_EINVAL, "invalid batch%s", "", 0);
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!ps[i]) return set_err(ADP_EINVAL, "null problem in batch at %s%lld", "", i);
        if (ps[i]->prm.prec != ps[0]->prm.prec || ps[i]->device != ps[0]->device)
            return set_err(ADP_EINVAL, "batched problems must share precision and device%s", "", 0);
    }
    adp_batch *bt = new adp_batch();
    bt->ps.assign(ps, ps + n);
    bt->n = n;
    bt->prec = ps[0]->prm.prec;
    bt->esize = ps[0]->esize;
    bt->ctx_bytes = bt->prec == ADP_F32 ? sizeof(Ctx<float>) : sizeof(Ctx<double>);
    bt->job_bytes = bt->prec == ADP_F32 ? sizeof(Job<float>) : sizeof(Job<double>);
    // one block shape for all: the fewest warps any problem allows, and the
    // largest shared-memory footprint at that width
    int nw = MAXNW;
    for (adp_problem *p : bt->ps) nw = std::min(nw, p->nw);
    bt->nw = nw;
    size_t smem = 0;
    for (adp_problem *p : bt->ps) {
        const Geom &g = p->g;
        const int tot = bt->prec == ADP_F32 ? Layout<float>(p->prm.C, p->prm.K, nw, g.wsm).total
                                            : Layout<double>(p->prm.C, p->prm.K, nw, g.wsm).total;
        smem = std::max(smem, (size_t)tot * bt->esize);
    }
    bt->smem = smem;
    adp_status st = ADP_OK;
#define CKB(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            st = set_err(e_ == cudaErrorMemoryAllocation ? ADP_ENOMEM : ADP_ECUDA, "%s (code %lld)", \
                         cudaGetErrorString(e_), (long long)e_);                             \
            batch_free(bt);                                                                  \
            return st;                                                                       \
        }                                                                                    \
    } while (0)
    CKB(cudaSetDevice(ps[0]->device));
    int nsm = 0, maxsmem = 0;
    CKB(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ps[0]->device));
    CKB(cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ps[0]->device));
    const void *fn = bt->prec == ADP_F32 ? kernel_f32_batched() : kernel_f64_batched();
    CKB(optin_dynamic_smem(fn, maxsmem));
    int occ = 0;
    CKB(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * nw, smem));
    bt->max_ctas = occ * nsm;
    if (bt->max_ctas < n) {
        batch_free(bt);
        return set_err(ADP_EINVAL, "a batch holds at most one problem per co-resident CTA (%s%lld)", "", occ * nsm);
    }
    long long cap = 0;
    for (adp_problem *p : bt->ps) cap += p->grid;
    if (cap < bt->max_ctas) bt->max_ctas = (int)cap;
    if (n == 1) {                  // the single-problem kernel with the problem's own launch shape
        bt->nw = ps[0]->nw;
        bt->smem = ps[0]->smem;
        bt->max_ctas = ps[0]->grid;
    }
    bt->work.resize(n);
    for (int i = 0; i < n; ++i) bt->work[i] = (double)ps[i]->g.nstrips * ps[i]->prm.K * ps[i]->prm.K;
    batch_partition(bt);
    CKB(cudaMalloc(&bt->dctx, n * bt->ctx_bytes));
    CKB(cudaMalloc(&bt->djob, n * bt->job_bytes));
    CKB(cudaMalloc((void **)&bt->dfirst, (n + 1) * sizeof(int)));
    CKB(cudaMalloc((void **)&bt->dbar, (size_t)n * kBarStride * sizeof(unsigned)));
    CKB(cudaMalloc((void **)&bt->dout, (size_t)n * sizeof(DevOut)));
    CKB(cudaMalloc((void **)&bt->dtot, (size_t)n * sizeof(MaidTotals)));
    CKB(cudaMallocHost((void **)&bt->hout, (size_t)n * sizeof(DevOut)));
    CKB(cudaMallocHost((void **)&bt->hctx, n * bt->ctx_bytes));
    CKB(cudaMallocHost((void **)&bt->hjob, n * bt->job_bytes));
    CKB(cudaEventCreate(&bt->ev0));
    CKB(cudaEventCreate(&bt->ev1));
#undef CKB
    *out = bt;
    return ADP_OK;
}

void adp_batch_destroy(adp_batch *bt)
{
    if (!bt) return;
    cudaSetDevice(bt->ps[0]->device);
    cudaStreamSynchronize(bt->ps[0]->stream);
    batch_free(bt);
}

int adp_batch_group_size(adp_batch *bt, int i)
{
    if (!bt || i < 0 || i >= bt->n) return -1;
    return bt->first[i + 1] - bt->first[i];
}

double adp_batch_last_kernel_ms(adp_batch *bt) { return bt ? (double)bt->last_ms : -1.0; }

adp_status adp_batch_maid_step(adp_batch *bt, adp_maid_state *st, void *const *b, void *const *x, void *const *q)
{
    if (!bt || !st || !b || !x || !q) return set_err(ADP_EINVAL, "null argument%s", "", 0);
    for (int i = 0; i < bt->n; ++i) {
        if (!b[i] || !x[i] || !q[i]) return set_err(ADP_EINVAL, "null data pointer for problem %s%lld", "", i);
        if (st[i].max_bt < 1 || st[i].max_rounds < 1 || st[i].ll_max_iters < 0 || st[i].cg_max_iters < 0)
            return set_err(ADP_EINVAL, "invalid MAID state for problem %s%lld", "", i);
    }
    cudaStream_t stream = bt->ps[0]->stream;
    CK(cudaSetDevice(bt->ps[0]->device));
    if (bt->prec == ADP_F32) batch_fill<float>(bt, st, b, x, q, false, 0);
    else batch_fill<double>(bt, st, b, x, q, false, 0);
    CK(cudaMemcpyAsync(bt->dctx, bt->hctx, bt->n * bt->ctx_bytes, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(bt->djob, bt->hjob, bt->n * bt->job_bytes, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(bt->dfirst, bt->first.data(), (bt->n + 1) * sizeof(int), cudaMemcpyHostToDevice, stream));
    CK(cudaEventRecord(bt->ev0, stream));
    adp_status ls = batch_launch(bt, stream);
    if (ls != ADP_OK) return ls;
    CK(cudaEventRecord(bt->ev1, stream));
    CK(cudaMemcpyAsync(bt->hout, bt->dout, bt->n * sizeof(DevOut), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    CK(cudaEventElapsedTime(&bt->last_ms, bt->ev0, bt->ev1));
    const adp_status rs = batch_report(bt, st, nullptr);
    batch_rebalance(bt);
    return rs;
}


adp_status adp_batch_maid_run_graph(adp_batch *bt, adp_maid_state *st, void *const *b, void *const *x,
                                    void *const *q, int max_steps, long long *totals)
{
    if (!bt || !st || !b || !x || !q || max_steps < 1) return set_err(ADP_EINVAL, "invalid argument%s", "", 0);
    for (int i = 0; i < bt->n; ++i)
        if (!b[i] || !x[i] || !q[i]) return set_err(ADP_EINVAL, "null data pointer for problem %s%lld", "", i);
    cudaStream_t stream = bt->ps[0]->stream;
    CK(cudaSetDevice(bt->ps[0]->device));
    if (bt->prec == ADP_F32) batch_fill<float>(bt, st, b, x, q, true, max_steps);
    else batch_fill<double>(bt, st, b, x, q, true, max_steps);
    CK(cudaMemcpyAsync(bt->dctx, bt->hctx, bt->n * bt->ctx_bytes, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(bt->djob, bt->hjob, bt->n * bt->job_bytes, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(bt->dfirst, bt->first.data(), (bt->n + 1) * sizeof(int), cudaMemcpyHostToDevice, stream));
    CK(cudaMemsetAsync(bt->dtot, 0, bt->n * sizeof(MaidTotals), stream));
    CK(cudaStreamSynchronize(stream));
    // the steps are captured once per run shape (steps, CTAs) on a private
    // stream (the legacy default stream cannot be captured) and replayed; the
    // launch records they read are uploaded above, before every replay
    adp_status res = ADP_OK;
    if (!bt->cs) CK(cudaStreamCreateWithFlags(&bt->cs, cudaStreamNonBlocking));
    // (a resident run reads its MAID state through maid_home, so the job's own
    // copy of the state, its last field, does not enter the comparison)
    const size_t jcmp = bt->prec == ADP_F32 ? offsetof(Job<float>, maid) : offsetof(Job<double>, maid);
    const bool same_records = bt->n > 1 || (bt->gctx.size() == bt->ctx_bytes + bt->job_bytes &&
                                            !memcmp(bt->gctx.data(), bt->hctx, bt->ctx_bytes) &&
                                            !memcmp(bt->gctx.data() + bt->ctx_bytes, bt->hjob, jcmp));
    if (!bt->gexec || bt->gsteps != max_steps || bt->ggrid != bt->first[bt->n] || !same_records) {
        if (bt->n == 1) {          // records captured by value: remember them
            bt->gctx.assign(bt->hctx, bt->hctx + bt->ctx_bytes);
            bt->gctx.insert(bt->gctx.end(), bt->hjob, bt->hjob + bt->job_bytes);
        }
        if (bt->gexec) { cudaGraphExecDestroy(bt->gexec); bt->gexec = nullptr; }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(bt->cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            res = batch_launch(bt, bt->cs);   // one launch runs up to max_steps upper iterations per problem
            cudaError_t e2 = cudaStreamEndCapture(bt->cs, &graph);
            if (res == ADP_OK && e2 != cudaSuccess)
                res = set_err(ADP_ECUDA, "graph capture: %s%lld", cudaGetErrorString(e2), 0);
        } else {
            res = set_err(ADP_ECUDA, "graph capture: %s%lld", cudaGetErrorString(e), 0);
        }
        if (res == ADP_OK) {
            e = cudaGraphInstantiate(&bt->gexec, graph, 0);
            if (e != cudaSuccess) {
                bt->gexec = nullptr;
                res = set_err(ADP_ECUDA, "graph instantiation: %s%lld", cudaGetErrorString(e), 0);
            }
        }
        if (graph) cudaGraphDestroy(graph);
        bt->gsteps = max_steps;
        bt->ggrid = bt->first[bt->n];
    }
    if (res == ADP_OK) {
        cudaEventRecord(bt->ev0, bt->cs);
        cudaError_t e = cudaGraphLaunch(bt->gexec, bt->cs);
        cudaEventRecord(bt->ev1, bt->cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(bt->cs);
        if (e != cudaSuccess) res = set_err(ADP_ECUDA, "graph launch: %s%lld", cudaGetErrorString(e), 0);
        else cudaEventElapsedTime(&bt->last_ms, bt->ev0, bt->ev1);
    }
    if (res != ADP_OK) return res;
    CK(cudaMemcpy(bt->hout, bt->dout, bt->n * sizeof(DevOut), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(bt->hjob, bt->djob, bt->n * bt->job_bytes, cudaMemcpyDeviceToHost));
    std::vector<MaidIn> state(bt->n);
    for (int i = 0; i < bt->n; ++i)
        memcpy(&state[i], bt->hjob + i * bt->job_bytes + (bt->prec == ADP_F32 ? offsetof(Job<float>, maid) : offsetof(Job<double>, maid)), sizeof(MaidIn));
    if (totals) {
        std::vector<MaidTotals> t(bt->n);
        CK(cudaMemcpy(t.data(), bt->dtot, bt->n * sizeof(MaidTotals), cudaMemcpyDeviceToHost));
        for (int i = 0; i < bt->n; ++i) {
            totals[4 * i] = t[i].fused_iters; totals[4 * i + 1] = t[i].conv_passes;
            totals[4 * i + 2] = t[i].upper_iters; totals[4 * i + 3] = t[i].accepted;
        }
    }
    adp_status rs = batch_report(bt, st, state.data());
    for (int i = 0; i < bt->n; ++i) {
        st[i].stopped = (st[i].eps_stop > 0 && st[i].eps <= st[i].eps_stop) || state[i].halted;
    }
    batch_rebalance(bt);
    return rs;
}

} // extern "C"
