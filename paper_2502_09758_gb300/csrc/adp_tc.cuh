// Host interface of the tensor-core (BF16 operands, FP32 accumulation)
// operator B x / B^T z of Eq. 2.4, implemented in adp_tc.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>

namespace adp {

constexpr int TC_KMAX = 33;   // kernel sizes whose Toeplitz bands fit one 64-column tile

struct TcPlan;
struct TcTimes {
    float prep_ms;   // BF16 conversion of the image and the kernel bands
    float corr_ms;   // the tensor-core correlation
};

// Workspace for one C x H x W image and a C x K x K kernel on `device`:
// the BF16 padded image, the bands and the tensor map over the image.
// Returns 0, or nonzero with a message in err.
int tc_plan_create(int C, int H, int W, int K, int device, TcPlan **out, char *err, int errlen);
void tc_plan_destroy(TcPlan *p);
// out = B x (transpose = false) or B^T x (true), all FP32 device pointers;
// ordered on s and complete on return.  *dev_status receives the kernel's
// status (ST_OK or ST_TIMEOUT).  Returns 0, or nonzero on a CUDA error.
int tc_apply(TcPlan *p, const float *b, const float *x, float *out, bool transpose, long long timeout_ns,
             cudaStream_t s, TcTimes *times, int *dev_status, char *err, int errlen);
int tc_grid(const TcPlan *p);

// BF16 tensor map with 128-byte swizzle over a 3-D array (defined with the
// other tensor-map code of the library)
int encode_bf16_swizzled_3d(void *base, const unsigned long long dims[3], const unsigned long long strides[2],
                            const unsigned box[3], CUtensorMap *map, char *err, int errlen);

} // namespace adp
