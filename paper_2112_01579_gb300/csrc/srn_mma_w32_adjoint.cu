// Tensor-core variants with the adjoint input gradient (Section 5) for hidden
// width 32: 14 Fourier rows / 16 latent channels and 12 / 8, SnakeAlt and
// sine; the shaded render and the point evaluation of density + gradient.
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_ADJOINT, 0, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SINE, SRN_SHADE_ADJOINT, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SNAKEALT, SRN_SHADE_ADJOINT, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SINE, SRN_SHADE_ADJOINT, 0, 0)
// density and adjoint gradient at given points (srn_density_grad on FP16 contexts)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SNAKEALT, kPointsAdj, 0, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SINE, kPointsAdj, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SNAKEALT, kPointsAdj, 0, 0)
SRN_MMA_INSTANTIATE(32, 12, 8, SRN_ACT_SINE, kPointsAdj, 0, 0)

}  // namespace mma
}  // namespace srn
