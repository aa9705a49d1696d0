// Register-FFT passes, F64, axis length 384.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 384)
SFRD_ADJ_INSTANTIATE(double, 384)
}  // namespace v2
}  // namespace sfrd
