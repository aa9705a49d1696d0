// Register-FFT passes, F32, axis length 384.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 384)
SFRD_ADJ_INSTANTIATE(float, 384)
}  // namespace v2
}  // namespace sfrd
