// Register-FFT passes, F64, axis length 256.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 256)
SFRD_ADJ_INSTANTIATE(double, 256)
}  // namespace v2
}  // namespace sfrd
