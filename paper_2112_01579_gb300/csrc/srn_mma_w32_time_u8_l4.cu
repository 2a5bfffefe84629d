// Tensor-core renders of the four-layer width-32 SnakeAlt density network
// with the direct time input or the 8-bit latent grid, a single latent grid,
// layer and output counts fixed at compile time.
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 1, 0, 4, 1)
SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 1, 4, 1)

}  // namespace mma
}  // namespace srn
