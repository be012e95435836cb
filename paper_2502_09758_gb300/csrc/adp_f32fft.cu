// float instantiation of the persistent engine with the FFT operator path
// compiled in (see adp_engine.cuh); used by problems after adp_set_fft.
#include "adp_engine.cuh"

namespace adp {
const void *kernel_f32_fft() { return (const void *)adp_kernel<float, true>; }
} // namespace adp
