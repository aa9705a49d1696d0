// Register-FFT passes, F32, axis length 256.
#include "adjoint.cuh"

namespace sfrd {
namespace v2 {
// the compile-time boundary-condition variants live in sfrd_v2_f32_256_{p,d,n}.cu
extern template cudaError_t col2_launch_bc<float, 256, SFRD_BC_PERIODIC>(const ColArgs<float>&, int, dim3, cudaStream_t);
extern template cudaError_t col2_launch_bc<float, 256, SFRD_BC_DIRICHLET>(const ColArgs<float>&, int, dim3, cudaStream_t);
extern template cudaError_t col2_launch_bc<float, 256, SFRD_BC_NEUMANN>(const ColArgs<float>&, int, dim3, cudaStream_t);
extern template cudaError_t x2_launch_bc<float, 256, SFRD_BC_PERIODIC>(const XArgs<float>&, int, dim3, cudaStream_t);
extern template cudaError_t x2_launch_bc<float, 256, SFRD_BC_DIRICHLET>(const XArgs<float>&, int, dim3, cudaStream_t);
extern template cudaError_t x2_launch_bc<float, 256, SFRD_BC_NEUMANN>(const XArgs<float>&, int, dim3, cudaStream_t);
extern template cudaError_t prepare2_bc<float, 256, SFRD_BC_PERIODIC>();
extern template cudaError_t prepare2_bc<float, 256, SFRD_BC_DIRICHLET>();
extern template cudaError_t prepare2_bc<float, 256, SFRD_BC_NEUMANN>();
SFRD_V2_INSTANTIATE(float, 256)
SFRD_ADJ_INSTANTIATE(float, 256)
}  // namespace v2
}  // namespace sfrd
