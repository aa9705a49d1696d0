// Register-FFT passes, FP32, axis length 128, compiled as five objects (SFRD_TU_PART 0-4): dispatch and
// plain column passes, element-pair stage passes, rational-coefficient stage passes, contiguous-axis
// pass, adjoint passes.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
#if SFRD_TU_PART == 0
SFRD_V2_EXTERN_FAMILIES(float, 128, -1)
SFRD_V2_DISPATCH(float, 128)
SFRD_V2_PLAIN(float, 128, -1)
#elif SFRD_TU_PART == 1
SFRD_V2_PAIR(float, 128, -1)
#elif SFRD_TU_PART == 2
SFRD_V2_RAT(float, 128, -1)
#elif SFRD_TU_PART == 3
SFRD_V2_X(float, 128, -1)
#elif SFRD_TU_PART == 4
SFRD_ADJ_INSTANTIATE(float, 128)
#endif
}  // namespace v2
}  // namespace sfrd
