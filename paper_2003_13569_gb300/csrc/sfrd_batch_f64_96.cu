// Batched persistent kernels, F64, register-engine axis length 96.
#include "batch_kernels.cuh"

namespace sfrd {
namespace v2 {
SFRD_BATCH_INSTANTIATE(double, 96)
}  // namespace v2
}  // namespace sfrd
