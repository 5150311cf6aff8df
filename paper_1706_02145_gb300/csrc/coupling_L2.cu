// Coupling kernel instantiation for lmax = 2 (FP64 and FP32).
#include "coupling_launch.cuh"

namespace celes {
CELES_INSTANTIATE_COUPLING(2, 1)
}  // namespace celes
