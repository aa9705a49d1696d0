// Batched persistent kernels, F32, register-engine axis length 512.
#include "batch_kernels.cuh"

namespace sfrd {
namespace v2 {
SFRD_BATCH_INSTANTIATE(float, 512)
}  // namespace v2
}  // namespace sfrd
