// FP32 CUDA-core render (no / finite-difference / head shading) and point
// evaluation for hidden width 48.
#include "srn_fp32_kernel.cuh"

namespace srn {
namespace fp32 {

SRN_FP32_RENDER(48, SRN_SHADE_NONE)
SRN_FP32_RENDER(48, SRN_SHADE_FD)
SRN_FP32_RENDER(48, SRN_SHADE_HEAD)
SRN_FP32_EVAL(48, 0)

}  // namespace fp32
}  // namespace srn
