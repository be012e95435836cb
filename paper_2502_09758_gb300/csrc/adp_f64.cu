// double instantiation of the persistent engine (see adp_engine.cuh).
#include "adp_engine.cuh"

namespace adp {
const void *kernel_f64() { return (const void *)adp_kernel<double>; }
} // namespace adp
