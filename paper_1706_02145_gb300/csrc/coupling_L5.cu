// Coupling kernel instantiation for lmax = 5 (FP32 unrolled; FP64 through the runtime-table kernel).
#include "coupling_launch.cuh"

namespace celes {
CELES_INSTANTIATE_COUPLING(5, 0)
}  // namespace celes
