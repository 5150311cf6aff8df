// Alternative FP32 coupling-kernel shape for lmax = 2 (an autotuner candidate).
#include "coupling_launch.cuh"

namespace celes {
CELES_INSTANTIATE_RTR_ALT(2)
}  // namespace celes
