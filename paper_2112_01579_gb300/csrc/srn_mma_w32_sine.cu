// Tensor-core render / point-evaluation variants for hidden width 32, 14 Fourier rows, 16 latent channels, sine activation.
#include "srn_mma_kernel.cuh"

namespace srn {
namespace mma {

SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SINE, SRN_SHADE_NONE, 0, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SINE, SRN_SHADE_FD, 0, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SINE, SRN_SHADE_HEAD, 0, 0)
SRN_MMA_INSTANTIATE(32, 14, 16, SRN_ACT_SINE, kPoints, 0, 0)

}  // namespace mma
}  // namespace srn
