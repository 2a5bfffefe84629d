// Dispatch of the FP32 CUDA-core render and point evaluation by hidden width
// and mode.  The kernels are in srn_fp32_kernel.cuh.
#include "srn_fp32.h"

namespace srn {
using fp32::launch_eval_t;
using fp32::launch_render_t;

bool render_fp32_supported(int width) { return width == 32 || width == 48 || width == 64; }

namespace {
template <int C>
cudaError_t render_width(const NetDev& net, const BatchDev& b, cudaStream_t s) {
  switch (b.shading) {
    case SRN_SHADE_NONE: return launch_render_t<C, SRN_SHADE_NONE>(net, b, s);
    case SRN_SHADE_ADJOINT: return launch_render_t<C, SRN_SHADE_ADJOINT>(net, b, s);
    case SRN_SHADE_FD: return launch_render_t<C, SRN_SHADE_FD>(net, b, s);
    default: return launch_render_t<C, SRN_SHADE_HEAD>(net, b, s);
  }
}
template <int C>
cudaError_t eval_width(const NetDev& net, const float* pts, int n, float time, float* out, float* grad,
                       const float* dout, int mode, cudaStream_t s) {
  if (mode == 0) return launch_eval_t<C, 0>(net, pts, n, time, out, grad, dout, s);
  if (mode == 1) return launch_eval_t<C, 1>(net, pts, n, time, out, grad, dout, s);
  return launch_eval_t<C, 2>(net, pts, n, time, out, grad, dout, s);
}
}  // namespace

cudaError_t launch_render_fp32(const NetDev& net, const BatchDev& b, cudaStream_t s) {
  if (net.c == 48) return render_width<48>(net, b, s);
  if (net.c == 64) return render_width<64>(net, b, s);
  return render_width<32>(net, b, s);
}

cudaError_t launch_eval_fp32(const NetDev& net, const float* pts, int n, float time, float* out, float* grad,
                             int mode, cudaStream_t s, const float* dout) {
  if (n == 0) return cudaSuccess;
  if (net.c == 48) return eval_width<48>(net, pts, n, time, out, grad, dout, mode, s);
  if (net.c == 64) return eval_width<64>(net, pts, n, time, out, grad, dout, mode, s);
  return eval_width<32>(net, pts, n, time, out, grad, dout, mode, s);
}

}  // namespace srn
