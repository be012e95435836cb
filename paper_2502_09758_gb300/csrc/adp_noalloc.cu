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
// image.
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
} // namespace adp

using namespace adp;

namespace {

// Layout of the scratch array: barrier counter | status/result record |
// reduction partials | five images (x_k, x_{k+1}, y_k, y_{k+1}, residual).
constexpr size_t kHeadBytes = 256;                                   // barrier counter
constexpr size_t kOutBytes = 256;                                    // DevOut
constexpr size_t kPartBytes = (size_t)NSLOT * GT_MAX * sizeof(double);
constexpr size_t kImages = 5;
constexpr size_t kImageBytes = ADP_NOALLOC_MAX_IMAGE_BYTES;
constexpr size_t kScratchBytes = kHeadBytes + kOutBytes + kPartBytes + kImages * kImageBytes;

static_assert(sizeof(DevOut) <= kOutBytes, "result record does not fit its slot");
static_assert(kScratchBytes == ADP_NOALLOC_SCRATCH_BYTES, "scratch layout and the size stated in adp.h differ");

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
        if (cudaFuncSetAttribute(kernel_f32(), cudaFuncAttributeMaxDynamicSharedMemorySize, s.maxsmem - 5 * 1024) !=
                cudaSuccess ||
            cudaFuncSetAttribute(kernel_f64(), cudaFuncAttributeMaxDynamicSharedMemorySize, s.maxsmem - 5 * 1024) !=
                cudaSuccess)
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
    constexpr int MR = Cfg<T>::MR;
    const int Kp = round_up(q.K, Cfg<T>::PC);
    const int nx = (q.W + 31) / 32, ny = (q.H + MR - 1) / MR, nstrips = q.C * nx * ny;
    int w_elems = 0, warp_elems = 0, total = 0, nw = MAXNW;
    for (; nw >= 1; --nw) {
        smem_layout<T>(q.C, q.K, nw, w_elems, warp_elems, total);
        if ((size_t)total * sizeof(T) + 5 * 1024 <= (size_t)ds.maxsmem) break;
    }
    if (nw < 1) return fail(ADP_EINVAL, "kernel size too large for shared memory");
    const size_t smem = (size_t)total * sizeof(T);
    const void *fn = sizeof(T) == 4 ? kernel_f32() : kernel_f64();
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * nw, smem) != cudaSuccess || occ < 1)
        return fail(ADP_ECUDA, "occupancy query failed");
    long long grid = nstrips <= (long long)ds.nsm * nw ? (nstrips < ds.nsm ? nstrips : ds.nsm)
                                                        : ((long long)nstrips + nw - 1) / nw;
    if (grid > (long long)occ * ds.nsm) grid = (long long)occ * ds.nsm;
    if (grid > GT_MAX) grid = GT_MAX;

    unsigned char *base = ds.scratch;
    Ctx<T> c;
    memset(&c, 0, sizeof c);
    c.C = q.C; c.H = q.H; c.W = q.W; c.K = q.K; c.r = (q.K - 1) / 2; c.Kp = Kp;
    c.nx = nx; c.ny = ny; c.nstrips = nstrips;
    c.PA = 32 + 2 * c.r; c.RA = MR + Kp - 1;
    c.trace = nullptr; c.trace_cap = 0;
    c.HW = (long long)q.H * q.W; c.N = c.HW * q.C;
    c.reg = q.reg; c.alpha = q.alpha; c.rp = q.reg_param; c.beta = q.beta; c.w0 = q.sobolev_w0;
    c.ddphi_max = q.reg == ADP_REG_QUAD ? 1.0 : 1.0 / q.reg_param;
    c.alphaT = (T)q.alpha; c.rpT = (T)q.reg_param; c.irpT = (T)(1.0 / q.reg_param);
    c.y = (const T *)y; c.a = nullptr;
    c.bar = (unsigned *)base;
    c.out = (DevOut *)(base + kHeadBytes);
    c.part = (double *)(base + kHeadBytes + kOutBytes);
    T *img = (T *)(base + kHeadBytes + kOutBytes + kPartBytes);
    const size_t stride = kImageBytes / sizeof(T);
    c.X0 = img; c.X1 = img + stride; c.Y0 = img + 2 * stride; c.Y1 = img + 3 * stride; c.U = img + 4 * stride;
    const double to = q.wait_timeout_s > 0 ? q.wait_timeout_s : 2.0;
    c.timeout_ns = (long long)(to * 1e9);

    Job<T> j;
    memset(&j, 0, sizeof j);
    j.mode = M_LOWER_SOLVE; j.b = (const T *)b; j.x = (const T *)x; j.xo = (T *)x;
    j.eps = eps; j.max_iters = max_iters;

    // what must start at zero: the barrier's arrival counter and the record
    // (its status word); the images are written before they are read
    if (cudaMemsetAsync(base, 0, kHeadBytes + kOutBytes, stream) != cudaSuccess)
        return fail(ADP_ECUDA, "clearing the scratch header failed");
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
    const size_t esize = q.prec == ADP_F32 ? sizeof(float) : sizeof(double);
    const size_t bytes = (size_t)q.C * q.H * q.W * esize;
    if (bytes > kImageBytes) {
        char msg[160];
        snprintf(msg, sizeof msg, "image of %zu bytes exceeds the no-allocation limit of %zu bytes (C*H*W*element size)",
                 bytes, (size_t)kImageBytes);
        return fail(ADP_EINVAL, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(ADP_ECUDA, "cudaGetDevice failed");
    DeviceSetup *ds = nullptr;
    adp_status st = setup_device(dev, &ds);
    if (st != ADP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return q.prec == ADP_F32 ? run_noalloc<float>(q, *ds, y, b, x, eps, max_iters, s, iters, gradnorm)
                             : run_noalloc<double>(q, *ds, y, b, x, eps, max_iters, s, iters, gradnorm);
}
