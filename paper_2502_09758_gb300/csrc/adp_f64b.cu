// double instantiation of the batched entry of the persistent engine (see
// adp_engine.cuh); a translation unit of its own so that it compiles in
// parallel with the single-problem entry.
#include "adp_engine.cuh"

namespace adp {
const void *kernel_f64_batched() { return (const void *)adp_kernel_batched<double>; }
} // namespace adp
