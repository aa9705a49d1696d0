// Register-FFT passes, F32, axis length 512.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 512)
SFRD_ADJ_INSTANTIATE(float, 512)
}  // namespace v2
}  // namespace sfrd
