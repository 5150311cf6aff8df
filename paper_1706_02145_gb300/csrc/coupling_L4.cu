// Coupling kernel instantiation for lmax = 4 (FP64 and FP32).
#include "coupling_launch.cuh"

namespace celes {
CELES_INSTANTIATE_COUPLING(4, 1)
}  // namespace celes
