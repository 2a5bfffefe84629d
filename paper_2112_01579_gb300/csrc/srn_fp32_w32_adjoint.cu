// FP32 CUDA-core render with adjoint gradient shading and the density +
// adjoint-gradient point evaluation for hidden width 32.
#include "srn_fp32_kernel.cuh"

namespace srn {
namespace fp32 {

SRN_FP32_RENDER(32, SRN_SHADE_ADJOINT)
SRN_FP32_EVAL(32, 1)
SRN_FP32_EVAL(32, 2)

}  // namespace fp32
}  // namespace srn
