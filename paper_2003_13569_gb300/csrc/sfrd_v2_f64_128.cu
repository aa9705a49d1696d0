// Register-FFT passes, F64, axis length 128.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 128)
SFRD_ADJ_INSTANTIATE(double, 128)
}  // namespace v2
}  // namespace sfrd
