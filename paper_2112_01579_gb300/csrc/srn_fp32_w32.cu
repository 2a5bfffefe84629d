// FP32 CUDA-core render (no / finite-difference / head shading) and point
// evaluation for hidden width 32.
#include "srn_fp32_kernel.cuh"

namespace srn {
namespace fp32 {

SRN_FP32_RENDER(32, SRN_SHADE_NONE)
SRN_FP32_RENDER(32, SRN_SHADE_FD)
SRN_FP32_RENDER(32, SRN_SHADE_HEAD)
SRN_FP32_EVAL(32, 0)

}  // namespace fp32
}  // namespace srn
