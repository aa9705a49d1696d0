// Batched persistent kernels, F32, register-engine axis length 64.
#include "batch_kernels.cuh"

namespace sfrd {
namespace v2 {
SFRD_BATCH_INSTANTIATE(float, 64)
}  // namespace v2
}  // namespace sfrd
