// The operator of Eq. 2.4 on the tensor cores: B x (or B^T z) with the image
// and the kernel rounded to BF16 and the products accumulated in FP32
// (tcgen05.mma kind::f16, accumulator in tensor memory).
//
// A correlation out[i,j] = sum_{p,q} w[p,q] x[i+p-r, j+q-r] is, for an output
// tile of TM = 128 rows x TN = 32 columns at (i0, j0), a sum over the kernel
// rows p of GEMMs
//   out[i0+m, j0+n] += sum_k A_p[m,k] T_p[n,k],
//   A_p[m,k] = x[i0+m+p-r, j0+k-r]   (k < KT = 64: the tile's input columns)
//   T_p[n,k] = w[p, k-n]             (zero unless 0 <= k-n < K: a Toeplitz band)
// A_p for every p is a row-shifted view of one staged image tile of TM+K-1
// rows, so the tile is loaded once (one TMA box, 128-byte swizzle) and each
// MMA's shared-memory descriptor starts p rows further down (the swizzle
// phase follows the address bits, so no base-offset correction).  The bands
// T_p of a channel are built once per call in global memory, already in the
// swizzled K-major layout, and copied into shared memory with one bulk copy
// when a CTA moves to a new channel.  B x correlates with the flipped kernel
// (Eq. 2.4), B^T z with the kernel as stored.  K <= 33 (TN + K - 1 <= KT).
//
// CTAs are persistent over (channel, tile) items in channel-major order, with
// warp roles: one thread issues the TMA copies into a ring of image slots, one
// issues the MMAs, and four warps read the accumulator (one output row per
// lane) and store the FP32 outputs.  Two accumulators alternate, so one
// tile's epilogue overlaps the next tile's MMAs.  Every wait is bounded; a
// wait that gives up records ST_TIMEOUT, stops the other roles, waits
// (bounded) for the CTA's own copies and MMAs still in flight, releases the
// tensor memory and returns.
#include "adp_device.cuh"
#include "adp_tc.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

namespace adp {

cudaError_t optin_dynamic_smem(const void *fn, int maxsmem);   // adp.cu

namespace {

constexpr int TM = 128, TN = 32, KT = 64;   // tile rows, tile columns, band width (BF16 elements)
constexpr int BAND_BYTES = TN * KT * 2;     // one band T_p: 32 rows of 128 bytes

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 1024 bytes
// between 8-row groups, descriptor version 1 (Blackwell)
__device__ __forceinline__ uint64_t sdesc(unsigned saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// x (FP32, C x H x W) -> BF16 image with periodic ghosts of r rows and r
// columns: xb[c][pi][pj] = x[c][(pi - r) mod H][(pj - r) mod W] for
// pi < H + 2r, pj < W + 2r; zero elsewhere (row pitch Wp, a multiple of 8;
// Hp rows).  One block row per padded row (blockIdx.y = c * Hp + pi); each
// thread writes 8 consecutive BF16 values with one 16-byte store.
__global__ void to_bf16_padded(const float *__restrict__ x, __nv_bfloat16 *__restrict__ xb, int H, int W, int r,
                               int Hp, int Wp)
{
    const int row = blockIdx.y, c = row / Hp, pi = row - c * Hp;
    int i = pi - r;
    const bool rin = pi < H + 2 * r;
    if (i < 0 || i >= H) i = ((i % H) + H) % H;
    const float *xr = x + ((long long)c * H + i) * W;
    uint4 *dst = reinterpret_cast<uint4 *>(xb + (long long)row * Wp);
    const int nv = Wp >> 3, wend = W + 2 * r;
    for (int v8 = blockIdx.x * blockDim.x + threadIdx.x; v8 < nv; v8 += gridDim.x * blockDim.x) {
        const int pj0 = v8 * 8;
        float f[8];
        if (rin && pj0 >= r && pj0 + 8 <= r + W) {   // interior: no wrap
#pragma unroll
            for (int e = 0; e < 8; ++e) f[e] = __ldg(xr + pj0 - r + e);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int pj = pj0 + e;
                f[e] = 0.f;
                if (rin && pj < wend) {
                    int j = pj - r;
                    if (j < 0 || j >= W) j = ((j % W) + W) % W;
                    f[e] = __ldg(xr + j);
                }
            }
        }
        uint4 o;
        __nv_bfloat162 h0 = __floats2bfloat162_rn(f[0], f[1]), h1 = __floats2bfloat162_rn(f[2], f[3]),
                       h2 = __floats2bfloat162_rn(f[4], f[5]), h3 = __floats2bfloat162_rn(f[6], f[7]);
        o.x = *reinterpret_cast<unsigned *>(&h0);
        o.y = *reinterpret_cast<unsigned *>(&h1);
        o.z = *reinterpret_cast<unsigned *>(&h2);
        o.w = *reinterpret_cast<unsigned *>(&h3);
        dst[v8] = o;
    }
}

// b (FP32, C x K x K) -> the swizzled bands of every channel: band (c, p) is
// 32 rows (output column n) x 64 BF16 (tile column k); element (n, k) sits
// at byte n*128 + (((2k)/16) ^ (n % 8))*16 + (2k) % 16 and holds w[p, k-n]
// (zero outside 0 <= k-n < K), w the flipped kernel (flip) or b itself.
__global__ void make_bands(const float *__restrict__ b, __nv_bfloat16 *__restrict__ bands, int C, int K, int flip)
{
    const long long n = (long long)C * K * TN * KT;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % KT);
        const long long t = e / KT;
        const int nn = (int)(t % TN);
        const long long cp = t / TN;
        const int p = (int)(cp % K), c = (int)(cp / K);
        const int q = k - nn;
        float v = 0.f;
        if (q >= 0 && q < K) {
            const float *bc = b + (long long)c * K * K;
            v = flip ? __ldg(bc + (K - 1 - p) * K + (K - 1 - q)) : __ldg(bc + p * K + q);
        }
        const int byte = nn * 128 + ((((2 * k) >> 4) ^ (nn & 7)) << 4) + ((2 * k) & 15);
        bands[cp * (BAND_BYTES / 2) + byte / 2] = __float2bfloat16_rn(v);
    }
}

__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t ad, uint64_t bd, unsigned idesc, unsigned acc)
{
    asm volatile("{\n .reg .pred pa;\n setp.ne.u32 pa, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(tmem),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mb)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mb))
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this warp's 32 lanes (one row
// per lane), waited for
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&f)[32])
{
    unsigned v[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                 "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) f[q] = __uint_as_float(v[q]);
}

// a bounded wait that also gives up as soon as another role has failed
__device__ __forceinline__ bool wait_or_fail(uint64_t *mb, unsigned parity, long long timeout_ns,
                                             volatile int *fail)
{
    if (mbar_try_wait(mb, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(mb, parity)) return true;
        if (*fail) return false;
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
            *fail = 1;
            return false;
        }
    }
}

// Warp roles: 0-3 read the accumulator and store the outputs (warp w owns
// tensor-memory lanes 32w..32w+31, i.e. output rows 32w..32w+31 of a tile);
// lane 0 of warp 4 issues the MMAs; lane 0 of warp 5 issues the copies.
// Image slots (NS of them) cycle through the CTA's tiles; the two
// accumulators (32 columns each) alternate between consecutive tiles, so one
// tile's epilogue overlaps the next tile's MMAs.
//   full[s]  image box of slot s landed          (copy -> MMA)
//   empty[s] the MMAs reading slot s completed    (MMA commit -> copy)
//   bfull    the current channel's bands landed   (copy -> MMA)
//   accf[a]  accumulator a holds a finished tile  (MMA commit -> epilogue)
//   acce[a]  accumulator a has been read          (4 epilogue warps -> MMA)
constexpr int NTHREADS = 192, NSMAX = 3;
// tensor-memory columns per CTA: the accumulators of two tiles in flight
constexpr int TMEM_COLS = 2 * TN;

__global__ void __launch_bounds__(NTHREADS, 1) tc_corr(const __grid_constant__ CUtensorMap xmap,
                                                       const __nv_bfloat16 *__restrict__ bands,
                                                       float *__restrict__ out, int C, int H, int W, int K, int NS,
                                                       long long timeout_ns, int *status)
{
    extern __shared__ unsigned char sm_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    const unsigned xbytes = (unsigned)(TM + K - 1) * 128u;
    const unsigned xslot = (xbytes + 1023u) / 1024u * 1024u;
    unsigned char *const bt = base + NS * xslot;
    __shared__ __align__(8) uint64_t full[NSMAX], empty[NSMAX], bfull, accf[2], acce[2];
    __shared__ unsigned tmem_base;
    __shared__ volatile int fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "n"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int s = 0; s < NSMAX; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&bfull, 1);
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], 4);
        }
        fence_mbar_init();
        fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    const int ty = (H + TM - 1) / TM, tx = (W + TN - 1) / TN, per = ty * tx;
    const long long ntiles = (long long)C * per;
    const long long G = gridDim.x;

    if (warp == 5) {
        if (lane == 0) {   // ---------------------------------------------- copies
            const unsigned bbytes = (unsigned)K * BAND_BYTES;
            int cur_c = -1, nbl = 0;
            long long n = 0;
            for (long long t = blockIdx.x; t < ntiles; t += G, ++n) {
                const int s = (int)(n % NS);
                const int c = (int)(t / per), rem = (int)(t - (long long)c * per);
                const int i0 = (rem / tx) * TM, j0 = (rem % tx) * TN;
                if (n >= NS && !wait_or_fail(&empty[s], (unsigned)((n / NS - 1) & 1), timeout_ns, &fail)) break;
                if (c != cur_c) {
                    // the previous tile's MMAs (the last readers of the bands) are complete
                    if (n >= 1 && !wait_or_fail(&empty[(n - 1) % NS], (unsigned)(((n - 1) / NS) & 1), timeout_ns,
                                                &fail))
                        break;
                    mbar_expect_tx(&bfull, bbytes);
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                 "[%3];" ::"r"(su32(bt)),
                                 "l"(bands + (long long)c * K * (BAND_BYTES / 2)), "r"(bbytes), "r"(su32(&bfull))
                                 : "memory");
                    cur_c = c;
                    ++nbl;
                }
                mbar_expect_tx(&full[s], xbytes);
                asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                             " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(base + s * xslot)),
                             "l"(&xmap), "r"(j0), "r"(i0), "r"(c), "r"(su32(&full[s]))
                             : "memory");
            }
            if (fail) {   // copies still in flight land before the CTA's memory goes away
                for (long long m = n - 1; m >= 0 && m >= n - NS; --m)
                    mbar_wait(&full[m % NS], (unsigned)((m / NS) & 1), timeout_ns);
                if (nbl > 0) mbar_wait(&bfull, (unsigned)((nbl - 1) & 1), timeout_ns);
            }
        }
    } else if (warp == 4) {
        if (lane == 0) {   // ---------------------------------------------- MMAs
            // instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N = TN, M = TM
            const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TN >> 3) << 17) |
                                   ((unsigned)(TM >> 4) << 24);
            const uint64_t bd0 = sdesc(su32(bt));
            int cur_c = -1, nbl = 0;
            long long n = 0, last = -1;
            for (long long t = blockIdx.x; t < ntiles; t += G, ++n) {
                const int s = (int)(n % NS), a = (int)(n & 1);
                const int c = (int)(t / per);
                if (!wait_or_fail(&full[s], (unsigned)((n / NS) & 1), timeout_ns, &fail)) break;
                if (c != cur_c) {
                    if (!wait_or_fail(&bfull, (unsigned)(nbl & 1), timeout_ns, &fail)) break;
                    ++nbl;
                    cur_c = c;
                }
                if (n >= 2 && !wait_or_fail(&acce[a], (unsigned)((n / 2 - 1) & 1), timeout_ns, &fail)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // descriptors advance by address / 16: a kernel row is one 128-byte
                // image row (+8) or one band (+BAND_BYTES/16), a k step 32 bytes (+2)
                const unsigned acc = tmem + (unsigned)(a * TN);
                const uint64_t ad0 = sdesc(su32(base + s * xslot));
                for (int p = 0; p < K; ++p) {
                    const uint64_t ad = ad0 + (uint64_t)(p * 8), bd = bd0 + (uint64_t)(p * (BAND_BYTES / 16));
#pragma unroll
                    for (int ks = 0; ks < KT / 16; ++ks)
                        mma_bf16(acc, ad + 2 * ks, bd + 2 * ks, idesc, (p | ks) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
                mma_commit(&accf[a]);
                last = n;
            }
            if (fail && last >= 0)   // the last MMAs finish before the tensor memory is released
                mbar_wait(&accf[last & 1], (unsigned)((last / 2) & 1), timeout_ns);
        }
    } else {               // ---------------------------------------------- epilogue
        long long n = 0;
        for (long long t = blockIdx.x; t < ntiles; t += G, ++n) {
            const int a = (int)(n & 1);
            const int c = (int)(t / per), rem = (int)(t - (long long)c * per);
            const int i0 = (rem / tx) * TM, j0 = (rem % tx) * TN;
            // the whole warp leaves together (the tensor-memory load below is warp-wide)
            const bool ok = wait_or_fail(&accf[a], (unsigned)((n / 2) & 1), timeout_ns, &fail);
            if (!__all_sync(0xffffffffu, ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float v[32];
            tmem_ld32(tmem + (unsigned)(a * TN) + ((unsigned)(warp * 32) << 16), v);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[a]);
            const int i = i0 + warp * 32 + lane;
            if (i < H) {
                float *orow = out + ((long long)c * H + i) * W + j0;
                if (j0 + TN <= W && ((reinterpret_cast<uintptr_t>(orow) & 15) == 0)) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        reinterpret_cast<float4 *>(orow)[q] =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < TN; ++q)
                        if (j0 + q < W) orow[q] = v[q];
                }
            }
        }
    }
    if (tid == 0 && fail) atomicCAS(status, ST_OK, ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
}

size_t tc_smem_bytes(int K, int NS)
{
    const size_t xslot = ((size_t)(TM + K - 1) * 128 + 1023) / 1024 * 1024;
    return 1024 + (size_t)NS * xslot + (size_t)K * BAND_BYTES;
}

} // namespace

struct TcPlan {
    int C, H, W, K, r, Hp, Wp, device, grid, NS;
    size_t smem;
    __nv_bfloat16 *xb, *bands;
    int *status, *hstatus;
    CUtensorMap map;
    cudaEvent_t e0, e1, e2;
};

void tc_plan_destroy(TcPlan *p)
{
    if (!p) return;
    if (p->xb) cudaFree(p->xb);
    if (p->bands) cudaFree(p->bands);
    if (p->status) cudaFree(p->status);
    if (p->hstatus) cudaFreeHost(p->hstatus);
    if (p->e0) cudaEventDestroy(p->e0);
    if (p->e1) cudaEventDestroy(p->e1);
    if (p->e2) cudaEventDestroy(p->e2);
    free(p);
}

int tc_plan_create(int C, int H, int W, int K, int device, TcPlan **out, char *err, int errlen)
{
    *out = nullptr;
    if (K < 1 || K > TC_KMAX || (K & 1) == 0) {
        snprintf(err, errlen, "tensor-core operator needs an odd K <= %d (got %d)", TC_KMAX, K);
        return 1;
    }
    TcPlan *p = (TcPlan *)calloc(1, sizeof(TcPlan));
    if (!p) {
        snprintf(err, errlen, "host allocation failed");
        return 2;
    }
    p->C = C; p->H = H; p->W = W; p->K = K; p->r = (K - 1) / 2; p->device = device;
    // rows and columns of the padded image: at least one TMA box in each
    // direction, so that a box never exceeds the tensor
    p->Hp = std::max(H + 2 * p->r, TM + K - 1);
    p->Wp = std::max(round_up(W + 2 * p->r, 8), KT);
    int maxsmem = 0;
    if (cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        snprintf(err, errlen, "cannot query shared memory");
        tc_plan_destroy(p);
        return 3;
    }
    // three image slots when they fit beside the bands, else two
    p->NS = tc_smem_bytes(K, NSMAX) + 1024 <= (size_t)maxsmem ? NSMAX : 2;
    p->smem = tc_smem_bytes(K, p->NS);
#define TCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            snprintf(err, errlen, "%s (code %d)", cudaGetErrorString(e_), (int)e_);              \
            tc_plan_destroy(p);                                                                   \
            return 3;                                                                             \
        }                                                                                         \
    } while (0)
    const size_t xbytes = (size_t)C * p->Hp * p->Wp * sizeof(__nv_bfloat16);
    TCK(cudaMalloc((void **)&p->xb, xbytes));
    TCK(cudaMalloc((void **)&p->bands, (size_t)C * K * BAND_BYTES));
    TCK(cudaMalloc((void **)&p->status, sizeof(int)));
    TCK(cudaMallocHost((void **)&p->hstatus, sizeof(int)));
    TCK(cudaEventCreate(&p->e0));
    TCK(cudaEventCreate(&p->e1));
    TCK(cudaEventCreate(&p->e2));
    TCK(cudaMemset(p->xb, 0, xbytes));
    // the device's whole opt-in size rather than this plan's: the attribute is
    // shared by every plan, and a smaller value set for a later plan (smaller K)
    // would make the launches of an earlier, larger one fail
    TCK(optin_dynamic_smem((const void *)tc_corr, maxsmem));
    int nsm = 0, occ = 0;
    TCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    TCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tc_corr, NTHREADS, p->smem));
#undef TCK
    if (occ < 1) {
        snprintf(err, errlen, "tensor-core correlation cannot be resident (%zu bytes of shared memory)", p->smem);
        tc_plan_destroy(p);
        return 1;
    }
    // each resident CTA holds TMEM_COLS of the SM's 512 tensor-memory columns
    occ = std::min(occ, 512 / TMEM_COLS);
    const long long ntiles = (long long)C * ((H + TM - 1) / TM) * ((W + TN - 1) / TN);
    p->grid = (int)std::min<long long>(ntiles, (long long)occ * nsm);
    // [channel][padded row][padded column], innermost first
    const unsigned long long dims[3] = {(unsigned long long)p->Wp, (unsigned long long)p->Hp,
                                        (unsigned long long)C};
    const unsigned long long strides[2] = {(unsigned long long)p->Wp * 2, (unsigned long long)p->Hp * p->Wp * 2};
    const unsigned box[3] = {(unsigned)KT, (unsigned)(TM + K - 1), 1u};
    if (encode_bf16_swizzled_3d(p->xb, dims, strides, box, &p->map, err, errlen)) {
        tc_plan_destroy(p);
        return 3;
    }
    *out = p;
    return 0;
}

int tc_apply(TcPlan *p, const float *b, const float *x, float *out, bool transpose, long long timeout_ns,
             cudaStream_t s, TcTimes *times, int *dev_status, char *err, int errlen)
{
#define TCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            snprintf(err, errlen, "%s (code %d)", cudaGetErrorString(e_), (int)e_);              \
            return 3;                                                                             \
        }                                                                                         \
    } while (0)
    TCK(cudaMemsetAsync(p->status, 0, sizeof(int), s));
    TCK(cudaEventRecord(p->e0, s));
    const long long nb = (long long)p->C * p->K * TN * KT;
    make_bands<<<(int)std::max(1LL, std::min(1024LL, (nb + 255) / 256)), 256, 0, s>>>(b, p->bands, p->C, p->K,
                                                                                    transpose ? 0 : 1);
    TCK(cudaGetLastError());
    to_bf16_padded<<<dim3((p->Wp / 8 + 255) / 256, p->C * p->Hp), 256, 0, s>>>(x, p->xb, p->H, p->W, p->r, p->Hp,
                                                                          p->Wp);
    TCK(cudaGetLastError());
    TCK(cudaEventRecord(p->e1, s));
    tc_corr<<<p->grid, NTHREADS, p->smem, s>>>(p->map, p->bands, out, p->C, p->H, p->W, p->K, p->NS, timeout_ns,
                                               p->status);
    TCK(cudaGetLastError());
    TCK(cudaEventRecord(p->e2, s));
    TCK(cudaMemcpyAsync(p->hstatus, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    TCK(cudaStreamSynchronize(s));
    if (times) {
        TCK(cudaEventElapsedTime(&times->prep_ms, p->e0, p->e1));
        TCK(cudaEventElapsedTime(&times->corr_ms, p->e1, p->e2));
    }
#undef TCK
    *dev_status = *p->hstatus;
    return 0;
}

int tc_grid(const TcPlan *p) { return p ? p->grid : 0; }

} // namespace adp
