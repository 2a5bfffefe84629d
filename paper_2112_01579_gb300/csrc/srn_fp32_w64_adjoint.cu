// FP32 CUDA-core render with adjoint gradient shading and the density +
// adjoint-gradient point evaluation for hidden width 64.
#include "srn_fp32_kernel.cuh"

namespace srn {
namespace fp32 {

SRN_FP32_RENDER(64, SRN_SHADE_ADJOINT)
SRN_FP32_EVAL(64, 1)
SRN_FP32_EVAL(64, 2)

}  // namespace fp32
}  // namespace srn
