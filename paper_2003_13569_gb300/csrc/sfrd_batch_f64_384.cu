// Batched persistent kernels, F64, register-engine axis length 384.
#include "batch_kernels.cuh"

namespace sfrd {
namespace v2 {
SFRD_BATCH_INSTANTIATE(double, 384)
}  // namespace v2
}  // namespace sfrd
