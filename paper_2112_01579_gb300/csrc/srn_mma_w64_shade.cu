// Tensor-core render variants with shading (Section 5: adjoint backward MMAs,
// finite differences, 4-output head) and the adjoint at given points, for
// hidden width 64 (30 Fourier rows, 16 latent channels, SnakeAlt).
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE(64, 30, 16, SRN_ACT_SNAKEALT, SRN_SHADE_ADJOINT, 0, 0)
SRN_MMA_INSTANTIATE(64, 30, 16, SRN_ACT_SNAKEALT, kPointsAdj, 0, 0)
SRN_MMA_INSTANTIATE(64, 30, 16, SRN_ACT_SNAKEALT, SRN_SHADE_FD, 0, 0)
SRN_MMA_INSTANTIATE(64, 30, 16, SRN_ACT_SNAKEALT, SRN_SHADE_HEAD, 0, 0)

}  // namespace mma
}  // namespace srn
