// Register-FFT passes, F64, axis length 96.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 96)
SFRD_ADJ_INSTANTIATE(double, 96)
}  // namespace v2
}  // namespace sfrd
