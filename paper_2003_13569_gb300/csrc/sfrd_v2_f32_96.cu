// Register-FFT passes, F32, axis length 96.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 96)
SFRD_ADJ_INSTANTIATE(float, 96)
}  // namespace v2
}  // namespace sfrd
