// Register-FFT passes, F32, axis length 128.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 128)
SFRD_ADJ_INSTANTIATE(float, 128)
}  // namespace v2
}  // namespace sfrd
