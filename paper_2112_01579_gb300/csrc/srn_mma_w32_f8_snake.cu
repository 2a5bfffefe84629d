// Tensor-core render / point-evaluation variants for hidden width 32, 12 Fourier rows, 8 latent channels, SnakeAlt.
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SNAKEALT, SRN_SHADE_FD, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SNAKEALT, SRN_SHADE_HEAD, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SNAKEALT, kPoints, 0, 0)

}  // namespace mma
}  // namespace srn
