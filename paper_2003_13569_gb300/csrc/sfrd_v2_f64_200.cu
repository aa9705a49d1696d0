// Register-FFT passes, F64, axis length 200.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 200)
SFRD_ADJ_INSTANTIATE(double, 200)
}  // namespace v2
}  // namespace sfrd
