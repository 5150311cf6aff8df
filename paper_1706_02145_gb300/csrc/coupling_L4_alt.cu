// Alternative FP32 coupling-kernel shape for lmax = 4 (an autotuner candidate).
#include "coupling_launch.cuh"

namespace celes {
CELES_INSTANTIATE_RTR_ALT(4)
}  // namespace celes
