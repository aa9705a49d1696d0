// Register-FFT passes, F64, axis length 512.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 512)
SFRD_ADJ_INSTANTIATE(double, 512)
}  // namespace v2
}  // namespace sfrd
