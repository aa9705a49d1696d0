// Register-FFT passes, FP32, axis length 200, compiled as five objects (SFRD_TU_PART 0-4): dispatch and
// plain column passes, element-pair stage passes, rational-coefficient stage passes, contiguous-axis
// pass, adjoint passes.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
#if SFRD_TU_PART == 0
SFRD_V2_EXTERN_FAMILIES(float, 200, -1)
SFRD_V2_DISPATCH(float, 200)
SFRD_V2_PLAIN(float, 200, -1)
#elif SFRD_TU_PART == 1
SFRD_V2_PAIR(float, 200, -1)
#elif SFRD_TU_PART == 2
SFRD_V2_RAT(float, 200, -1)
#elif SFRD_TU_PART == 3
SFRD_V2_X(float, 200, -1)
#elif SFRD_TU_PART == 4
SFRD_ADJ_INSTANTIATE(float, 200)
#endif
}  // namespace v2
}  // namespace sfrd
