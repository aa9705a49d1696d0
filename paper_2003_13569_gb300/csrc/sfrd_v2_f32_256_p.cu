// Register-FFT passes, FP32, axis length 256, boundary condition fixed at compile time.
#include "passes2.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE_BC(float, 256, SFRD_BC_PERIODIC)
}  // namespace v2
}  // namespace sfrd
