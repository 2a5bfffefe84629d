// Tensor-core render variants with adjoint gradient shading (Section 5) for
// hidden width 32: 14 Fourier rows / 16 latent channels and 12 / 8, SnakeAlt
// and sine.
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_ADJOINT, 0, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SINE, SRN_SHADE_ADJOINT, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SNAKEALT, SRN_SHADE_ADJOINT, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SINE, SRN_SHADE_ADJOINT, 0, 0)

}  // namespace mma
}  // namespace srn
