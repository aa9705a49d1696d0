// Register-FFT passes, F32, axis length 64.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 64)
SFRD_ADJ_INSTANTIATE(float, 64)
}  // namespace v2
}  // namespace sfrd
