// Tensor-core render / point-evaluation variants for hidden width 32, 14 Fourier rows, 16 latent channels, SnakeAlt, with the direct time input (Section 7) or the 8-bit latent grid (Section 4.2).
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 1, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 1, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 1)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 0, 1)

}  // namespace mma
}  // namespace srn
