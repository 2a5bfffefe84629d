// Declarations of the FP32 CUDA-core kernel variants (srn_fp32_kernel.cuh),
// explicitly instantiated per hidden width and mode in srn_fp32_w*.cu so the
// variants compile in parallel; srn_fp32.cu dispatches.
#pragma once
#include "srn_internal.h"

namespace srn {
namespace fp32 {

template <int C, int SH>
cudaError_t launch_render_t(const NetDev& net, const BatchDev& b, cudaStream_t s);

template <int C, int MODE>
cudaError_t launch_eval_t(const NetDev& net, const float* pts, int n, float time, float* out, float* grad,
                          const float* dout, cudaStream_t s);

}  // namespace fp32
}  // namespace srn
