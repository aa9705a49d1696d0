// FP64 instantiation of the transform passes.
#include "passes.cuh"

namespace sfrd {
SFRD_INSTANTIATE(double)
}
