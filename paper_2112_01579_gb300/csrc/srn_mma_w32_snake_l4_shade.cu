// Shaded tensor-core renders (central differences, 4-output head) of
// the four-layer width-32 SnakeAlt network (14 Fourier rows, 16 latent
// channels) with a single latent grid, layer count and output count fixed
// at compile time.
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_FD, 0, 0, 4, 1)
SRN_MMA_INSTANTIATE_L(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_HEAD, 0, 0, 4, 1)

}  // namespace mma
}  // namespace srn
