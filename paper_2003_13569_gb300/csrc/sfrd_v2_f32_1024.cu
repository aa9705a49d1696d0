// Register-FFT passes, F32, axis length 1024.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(float, 1024)
SFRD_ADJ_INSTANTIATE(float, 1024)
}  // namespace v2
}  // namespace sfrd
