// Batched persistent kernels, F64, register-engine axis length 256.
#include "batch_kernels.cuh"

namespace sfrd {
namespace v2 {
SFRD_BATCH_INSTANTIATE(double, 256)
}  // namespace v2
}  // namespace sfrd
