// Batched persistent kernels, F32, register-engine axis length 96.
#include "batch_kernels.cuh"

namespace sfrd {
namespace v2 {
SFRD_BATCH_INSTANTIATE(float, 96)
}  // namespace v2
}  // namespace sfrd
