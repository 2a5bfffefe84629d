// Tensor-core render and point evaluation of the four-layer width-32
// SnakeAlt density network (14 Fourier rows, 16 latent channels, one output)
// with layer count and output fixed at compile time, so the layer loop
// unrolls; with a single latent grid (no keyframes) or with keyframes.
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 0, 4, 1)
SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 0, 4, 0)
SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0, 4, 1)
SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0, 4, 0)

}  // namespace mma
}  // namespace srn
