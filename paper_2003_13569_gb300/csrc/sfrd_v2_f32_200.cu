// Register-FFT passes, F32, axis length 200.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 200)
SFRD_ADJ_INSTANTIATE(float, 200)
}  // namespace v2
}  // namespace sfrd
