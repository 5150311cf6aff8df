// Coupling kernel instantiation for lmax = 1 (FP64 and FP32).
#include "coupling_launch.cuh"

namespace celes {
CELES_INSTANTIATE_COUPLING(1, 1)
}  // namespace celes
