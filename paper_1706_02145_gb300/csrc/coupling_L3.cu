// Coupling kernel instantiation for lmax = 3 (FP64 and FP32).
#include "coupling_launch.cuh"

namespace celes {
CELES_INSTANTIATE_COUPLING(3, 1)
}  // namespace celes
