// Register-FFT passes, F64, axis length 1024.
#include "passes2.cuh"

namespace sfrd {
namespace v2 {
SFRD_V2_INSTANTIATE(double, 1024)
}  // namespace v2
}  // namespace sfrd
