// Register-FFT passes, F32, axis length 256.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 256)
SFRD_ADJ_INSTANTIATE(float, 256)
}  // namespace v2
}  // namespace sfrd
