// FP32 instantiation of the transform passes (FP64-computed tables and coefficients).
#include "passes.cuh"

namespace sfrd {
SFRD_INSTANTIATE(float)
}
