// Tensor-core render / point-evaluation variants for hidden widths 48 and 64 (22 and 30 Fourier rows, 16 latent channels, SnakeAlt).
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE(48, 22, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 0)
SRN_MMA_INSTANTIATE(48, 22, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0)
SRN_MMA_INSTANTIATE(64, 30, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 0)
SRN_MMA_INSTANTIATE(64, 30, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0)

}  // namespace mma
}  // namespace srn
