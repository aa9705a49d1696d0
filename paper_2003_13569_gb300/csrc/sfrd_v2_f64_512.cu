// Register-FFT passes, FP64, axis length 512, compiled as five objects (SFRD_TU_PART 0-4): dispatch and
// plain column passes, element-pair stage passes, rational-coefficient stage passes, contiguous-axis
// pass, adjoint passes.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
#if SFRD_TU_PART == 0
SFRD_V2_EXTERN_FAMILIES(double, 512, -1)
SFRD_V2_DISPATCH(double, 512)
SFRD_V2_PLAIN(double, 512, -1)
#elif SFRD_TU_PART == 1
SFRD_V2_PAIR(double, 512, -1)
#elif SFRD_TU_PART == 2
SFRD_V2_RAT(double, 512, -1)
#elif SFRD_TU_PART == 3
SFRD_V2_X(double, 512, -1)
#elif SFRD_TU_PART == 4
SFRD_ADJ_INSTANTIATE(double, 512)
#endif
}  // namespace v2
}  // namespace sfrd
