// Register-FFT passes, F64, axis length 64.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 64)
SFRD_ADJ_INSTANTIATE(double, 64)
}  // namespace v2
}  // namespace sfrd
