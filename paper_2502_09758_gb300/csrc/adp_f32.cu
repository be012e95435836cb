// float instantiation of the persistent engine (see adp_engine.cuh).
#include "adp_engine.cuh"

namespace adp {
const void *kernel_f32() { return (const void *)adp_kernel<float>; }
} // namespace adp
