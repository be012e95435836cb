// adp_lower_solve_noalloc: the lower-level solve without any device allocation.
//
// Some callers cannot call cudaMalloc/cudaFree at the point where they need a
// solve: cudaFree synchronises the whole device, a caller running inside a
// latency-critical loop or a real-time pipeline cannot afford that, and
// callers that hand all device memory to their own pool allocator (or run
// under a hard memory budget fixed at start-up) must not have a library
// allocate behind their back.  This entry point therefore takes its workspace
// from one fixed, file-scope device array instead of adp_problem_create's
// cudaMalloc'd buffers.  The caller still passes the inputs and the in/out
// image.  Padded images of at most ADP_NOALLOC_MAX_IMAGE_BYTES are supported.
//
// The array lives in this file; device code never names it.  Host code may not
// use its name as an address (on the host it is only a stand-in), so the
// device address is looked up once per device with cudaGetSymbolAddress while
// that device is current, and passed to the kernel as plain pointers.
#include "adp_device.cuh"
#include "adp.h"

#include <cuda_runtime.h>
#include <mutex>
#include <stdio.h>
#include <string.h>

namespace adp {
const void *kernel_f32();
const void *kernel_f64();
void record_error(const char *msg);   // adp.cu: the message adp_last_error returns
cudaError_t optin_dynamic_smem(const void *fn, int maxsmem);   // adp.cu
} // namespace adp

using namespace adp;

namespace {

// Layout of the scratch array: barrier counter | status/result record |
// reduction partials | kernel weight slots | the padded images of a lower
// solve (y, x_k, x_{k+1}, y_k, y_{k+1}, residual, solution).
constexpr size_t kHeadBytes = 256;                                   // barrier counter
constexpr size_t kOutBytes = 256;                                    // DevOut
constexpr size_t kPartBytes = (size_t)NSLOT * GT_MAX * sizeof(double);
constexpr size_t kWeightBytes = ADP_NOALLOC_WEIGHT_BYTES;
constexpr size_t kImages = NBUF_LOWER;
constexpr size_t kImageBytes = ADP_NOALLOC_MAX_IMAGE_BYTES;
constexpr size_t kScratchBytes = kHeadBytes + kOutBytes + kPartBytes + kWeightBytes + kImages * kImageBytes;

static_assert(sizeof(DevOut) <= kOutBytes, "result record does not fit its slot");
static_assert(kScratchBytes == ADP_NOALLOC_SCRATCH_BYTES, "scratch layout and the size stated in adp.h differ");
static_assert(kImages == 7, "adp.h states seven images");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool ready;
    unsigned char *scratch;   // device address of g_scratch on this device
    int nsm, maxsmem;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

adp_status fail(adp_status s, const char *msg)
{
    record_error(msg);
    return s;
}

// Once per device, with that device current: the scratch address, SM count,
// shared-memory limit, and the kernels' dynamic shared-memory opt-in.
adp_status setup_device(int dev, DeviceSetup **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(ADP_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) return fail(ADP_ECUDA, "cudaGetSymbolAddress failed for the scratch array");
        if (cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&s.maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return fail(ADP_ECUDA, "device attribute query failed");
        if (optin_dynamic_smem(kernel_f32(), s.maxsmem) != cudaSuccess ||
            optin_dynamic_smem(kernel_f64(), s.maxsmem) != cudaSuccess)
            return fail(ADP_ECUDA, "cudaFuncSetAttribute failed");
        s.scratch = (unsigned char *)ptr;
        s.ready = true;
    }
    *out = &s;
    return ADP_OK;
}

template <typename T>
adp_status run_noalloc(const adp_params &q, DeviceSetup &ds, const void *y, const void *b, void *x, double eps,
                       int max_iters, cudaStream_t stream, int *iters, double *gradnorm)
{
    constexpr int MR = Cfg<T>::MR, NX = Cfg<T>::PC + MR - 1;
    const Geom g = make_geom<T>(q.C, q.H, q.W, q.K);
    const size_t img_bytes = (size_t)g.Np * sizeof(T);
    if (img_bytes > kImageBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "padded image of %zu bytes exceeds the no-allocation limit of %zu bytes (C*(H+2*Gy)*Wp*element size)",
                 img_bytes, (size_t)kImageBytes);
        return fail(ADP_EINVAL, msg);
    }
    if ((size_t)4 * q.C * q.K * g.Kp * sizeof(T) > kWeightBytes)
        return fail(ADP_EINVAL, "kernel weights exceed the no-allocation limit (4*C*K*Kp*element size)");
    int total = 0, nw = MAXNW;
    for (; nw >= 2; nw -= 2) {   // warps work in pairs
        total = Layout<T>(q.C, q.K, nw, g.wsm).total;
        if ((size_t)total * sizeof(T) + SMEM_STATIC_MARGIN <= (size_t)ds.maxsmem) break;
    }
    if (nw < 2) return fail(ADP_EINVAL, "kernel size too large for shared memory");
    const size_t smem = (size_t)total * sizeof(T);
    const void *fn = sizeof(T) == 4 ? kernel_f32() : kernel_f64();
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * nw, smem) != cudaSuccess || occ < 1)
        return fail(ADP_ECUDA, "occupancy query failed");
    long long grid = g.nstrips <= (long long)ds.nsm * nw ? (g.nstrips < ds.nsm ? g.nstrips : ds.nsm)
                                                          : ((long long)g.nstrips + nw - 1) / nw;
    if (grid > (long long)occ * ds.nsm) grid = (long long)occ * ds.nsm;
    if (grid > GT_MAX) grid = GT_MAX;

    unsigned char *base = ds.scratch;
    unsigned char *img = base + kHeadBytes + kOutBytes + kPartBytes + kWeightBytes;
    Ctx<T> c;
    memset(&c, 0, sizeof c);
    {
        char emsg[200];
        if (encode_tensor_maps(img, NBUF_LOWER, q.C, g, (int)sizeof(T), MR, NX, &c.map_s, &c.map_1, &c.map_i, emsg,
                               sizeof emsg))
            return fail(ADP_ECUDA, emsg);
    }
    c.C = q.C; c.H = q.H; c.W = q.W; c.K = q.K; c.r = g.r; c.Kp = g.Kp;
    c.r4 = g.r4; c.Gx = g.Gx; c.Gy = g.Gy; c.Wp = g.Wp; c.Hp = g.Hp; c.BW = g.BW;
    c.nx = g.nx; c.ny = g.ny; c.nstrips = g.nstrips; c.wsm = g.wsm; c.multiwrap = g.multiwrap;
    c.N = g.N; c.HW = g.HW; c.HWp = g.HWp; c.Np = g.Np;
    c.trace = nullptr; c.trace_cap = 0;
    c.reg = q.reg; c.alpha = q.alpha; c.rp = q.reg_param; c.beta = q.beta; c.w0 = q.sobolev_w0;
    c.ddphi_max = q.reg == ADP_REG_QUAD ? 1.0 : 1.0 / q.reg_param;
    c.alphaT = (T)q.alpha; c.rpT = (T)q.reg_param; c.irpT = (T)(1.0 / q.reg_param);
    c.a = nullptr;
    c.bar = (unsigned *)base;
    c.out = (DevOut *)(base + kHeadBytes);
    c.part = (double *)(base + kHeadBytes + kOutBytes);
    c.wg = (T *)(base + kHeadBytes + kOutBytes + kPartBytes);
    c.ws = (T *)img;
    const double to = q.wait_timeout_s > 0 ? q.wait_timeout_s : 2.0;
    c.timeout_ns = (long long)(to * 1e9);

    Job<T> j;
    memset(&j, 0, sizeof j);
    j.mode = M_LOWER_SOLVE; j.b = (const T *)b; j.x = (const T *)x; j.xo = (T *)x; j.y = (const T *)y;
    j.eps = eps; j.max_iters = max_iters;

    // what must start at zero: the barrier's arrival counter, the record (its
    // status word) and the images (their padding columns are read, never
    // written); the weights are written before they are read
    if (cudaMemsetAsync(base, 0, kHeadBytes + kOutBytes, stream) != cudaSuccess ||
        cudaMemsetAsync(img, 0, NBUF_LOWER * img_bytes, stream) != cudaSuccess)
        return fail(ADP_ECUDA, "clearing the scratch failed");
    void *args[] = {(void *)&c, (void *)&j};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(32 * nw), args, smem, stream);
    if (e != cudaSuccess) return fail(ADP_ECUDA, cudaGetErrorString(e));
    DevOut o;
    if (cudaMemcpyAsync(&o, c.out, sizeof o, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(ADP_ECUDA, "reading the result record failed");
    if (o.status == ST_TIMEOUT) return fail(ADP_ETIMEOUT, "device-side wait gave up");
    if (o.status == ST_NONFINITE) return fail(ADP_ENONFINITE, "non-finite value in a reduction");
    if (o.status != ST_OK) return fail(ADP_ECUDA, "unexpected device status");
    if (iters) *iters = o.iters;
    if (gradnorm) *gradnorm = o.gradnorm;
    return o.capped ? ADP_ENOCONV : ADP_OK;
}

} // namespace

extern "C" adp_status adp_lower_solve_noalloc(const adp_params *params, const void *y, const void *b, void *x,
                                              double eps, int max_iters, void *stream, int *iters,
                                              double *gradnorm)
{
    if (!params || !y || !b || !x) return fail(ADP_EINVAL, "null argument");
    const adp_params &q = *params;
    if (q.C < 1 || q.C > MAXC || q.H < 1 || q.W < 1) return fail(ADP_EINVAL, "bad image shape");
    if (q.K < 1 || q.K > KMAX || (q.K % 2) == 0) return fail(ADP_EINVAL, "K must be odd and in [1, 63]");
    if (q.prec != ADP_F32 && q.prec != ADP_F64) return fail(ADP_EINVAL, "unsupported precision");
    if (q.reg < 0 || q.reg > 2 || (q.reg != ADP_REG_QUAD && !(q.reg_param > 0)) || !(q.alpha >= 0))
        return fail(ADP_EINVAL, "bad regulariser parameters");
    if (max_iters < 0) return fail(ADP_EINVAL, "max_iters must be >= 0");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(ADP_ECUDA, "cudaGetDevice failed");
    DeviceSetup *ds = nullptr;
    adp_status st = setup_device(dev, &ds);
    if (st != ADP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return q.prec == ADP_F32 ? run_noalloc<float>(q, *ds, y, b, x, eps, max_iters, s, iters, gradnorm)
                             : run_noalloc<double>(q, *ds, y, b, x, eps, max_iters, s, iters, gradnorm);
}
