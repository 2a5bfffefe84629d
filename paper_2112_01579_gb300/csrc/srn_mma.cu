// Dispatch of the FP16 tensor-core render / point evaluation: which network
// shapes and shading modes have a kernel variant, and which variant runs.
// The kernel itself is in srn_mma_kernel.cuh.
#include <string.h>

#include "srn_mma.h"

namespace srn {
using mma::kPoints;
using mma::kPointsAdj;
using mma::launch_t;
using mma::PointsDev;

namespace {

template <int C, int M, int F, int ACT>
cudaError_t dispatch_shading(const NetDev& net, const BatchDev& b, unsigned long long* ctr, unsigned int* st,
                             cudaStream_t s) {
  switch (b.shading) {
    case SRN_SHADE_NONE: return launch_t<C, M, F, ACT, SRN_SHADE_NONE, 0, 0>(net, b, PointsDev{}, ctr, st, s);
    case SRN_SHADE_FD: return launch_t<C, M, F, ACT, SRN_SHADE_FD, 0, 0>(net, b, PointsDev{}, ctr, st, s);
    case SRN_SHADE_ADJOINT: return launch_t<C, M, F, ACT, SRN_SHADE_ADJOINT, 0, 0>(net, b, PointsDev{}, ctr, st, s);
    default: return launch_t<C, M, F, ACT, SRN_SHADE_HEAD, 0, 0>(net, b, PointsDev{}, ctr, st, s);
  }
}

// Shared memory the kernel needs for this network and shading (0: the shape
// is not tiled).
int mma_smem_bytes(const NetDev& n, int shading) {
  if (n.c != 32 && n.c != 48 && n.c != 64) return 0;
  const int sh = shading == SRN_SHADE_ADJOINT ? SRN_SHADE_ADJOINT : SRN_SHADE_NONE;  // the most warpgroups otherwise
  return mma::make_plan(n, n.c, mma::wgs_for(n.c, sh), sh == SRN_SHADE_ADJOINT).total;
}

}  // namespace

bool render_mma_supported(const NetDev& n, int shading) {
  if (n.l < 2 || n.l > 8) return false;
  // adjoint: backward MMAs, at most four layers (two stashed derivative
  // blocks in TMEM), no time input, FP16 grid; the gradient is that of
  // output 0, so the 4-output head is taken too
  if (shading == SRN_SHADE_ADJOINT && !(n.l <= mma::kAdjMaxLayers && !n.ti && !n.gq)) return false;
  if (shading == SRN_SHADE_HEAD && n.D != 4) return false;
  if (n.ti && !(n.c == 32 && n.m == 14 && n.F == 16 && n.act == SRN_ACT_SNAKEALT && shading == SRN_SHADE_NONE))
    return false;
  if (n.gq && !(n.c == 32 && n.m == 14 && n.F == 16 && n.act == SRN_ACT_SNAKEALT && shading == SRN_SHADE_NONE &&
                !n.ti))
    return false;
  const bool shape_a = n.c == 32 && n.m == 14 && n.F == 16;
  const bool shape_b = n.c == 32 && n.m == 12 && n.F == 8;
  // widths 48 / 64: the sweep's inputs (22 / 30 Fourier rows, 16 latent channels), SnakeAlt, every shading
  const bool shape_c = n.c == 48 && n.m == 22 && n.F == 16 && n.act == SRN_ACT_SNAKEALT;
  const bool shape_d = n.c == 64 && n.m == 30 && n.F == 16 && n.act == SRN_ACT_SNAKEALT;
  if (!shape_a && !shape_b && !shape_c && !shape_d) return false;
  const int smem = mma_smem_bytes(n, shading);
  if (smem == 0 || smem > 227 * 1024) return false;
  if ((size_t)n.nkey * n.R * n.R * n.R * n.F >= (size_t)1 << 31) return false;
  return n.act == SRN_ACT_SINE || n.act == SRN_ACT_SNAKEALT;
}

cudaError_t launch_render_mma(const NetDev& n, const BatchDev& b, unsigned long long* ctr, unsigned int* status,
                              cudaStream_t s) {
  // direct time input / 8-bit grid: the four-layer density network with a
  // single latent grid runs the specialised instantiation (see below)
  const bool l4s = n.l == 4 && n.D == 1 && n.nkey == 1;
  if (n.ti)
    return l4s ? launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 1, 0, 4, 1>(n, b, PointsDev{}, ctr, status, s)
               : launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 1, 0>(n, b, PointsDev{}, ctr, status, s);
  if (n.gq)
    return l4s ? launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 1, 4, 1>(n, b, PointsDev{}, ctr, status, s)
               : launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 1>(n, b, PointsDev{}, ctr, status, s);
  if (n.c == 48) return dispatch_shading<48, 22, 16, SRN_ACT_SNAKEALT>(n, b, ctr, status, s);
  if (n.c == 64) return dispatch_shading<64, 30, 16, SRN_ACT_SNAKEALT>(n, b, ctr, status, s);
  if (n.m == 14 && n.F == 16) {
    // the four-layer SnakeAlt networks of the inference and shading workloads:
    // layer loop unrolled, output count fixed and, for a single latent grid,
    // no time blend in the gather (the adjoint keeps the generic kernel, whose
    // register allocation spills less there)
    if (n.act == SRN_ACT_SNAKEALT && n.l == 4) {
      const PointsDev pd{};
      const bool st = n.nkey == 1;
      if (n.D == 1 && b.shading == SRN_SHADE_NONE)
        return st ? launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 0, 4, 1>(n, b, pd, ctr, status, s)
                  : launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_NONE, 0, 0, 4, 0>(n, b, pd, ctr, status, s);
      if (st && n.D == 1 && b.shading == SRN_SHADE_FD)
        return launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_FD, 0, 0, 4, 1>(n, b, pd, ctr, status, s);
      if (st && n.D == 4 && b.shading == SRN_SHADE_HEAD)
        return launch_t<32, 14, 16, SRN_ACT_SNAKEALT, SRN_SHADE_HEAD, 0, 0, 4, 1>(n, b, pd, ctr, status, s);
    }
    return n.act == SRN_ACT_SNAKEALT ? dispatch_shading<32, 14, 16, SRN_ACT_SNAKEALT>(n, b, ctr, status, s)
                                     : dispatch_shading<32, 14, 16, SRN_ACT_SINE>(n, b, ctr, status, s);
  }
  return n.act == SRN_ACT_SNAKEALT ? dispatch_shading<32, 12, 8, SRN_ACT_SNAKEALT>(n, b, ctr, status, s)
                                   : dispatch_shading<32, 12, 8, SRN_ACT_SINE>(n, b, ctr, status, s);
}

bool eval_mma_supported(const NetDev& n) { return render_mma_supported(n, SRN_SHADE_NONE); }

// Network output at n points with the tensor-core layers (mode kPoints).
cudaError_t launch_eval_mma(const NetDev& n, const float* pts, long long count, float time, float* out,
                            unsigned long long* ctr, unsigned int* status, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  BatchDev b;
  memset(&b, 0, sizeof(b));
  b.tf.n = 2;
  PointsDev pd{pts, out, count, time, nullptr};
  if (n.ti) return launch_t<32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 1, 0>(n, b, pd, ctr, status, s);
  if (n.gq) return launch_t<32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 0, 1>(n, b, pd, ctr, status, s);
  if (n.c == 48) return launch_t<48, 22, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0>(n, b, pd, ctr, status, s);
  if (n.c == 64) return launch_t<64, 30, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0>(n, b, pd, ctr, status, s);
  if (n.m == 14 && n.F == 16) {
    if (n.act == SRN_ACT_SNAKEALT && n.l == 4 && n.D == 1)
      return n.nkey == 1 ? launch_t<32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0, 4, 1>(n, b, pd, ctr, status, s)
                         : launch_t<32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0, 4, 0>(n, b, pd, ctr, status, s);
    return n.act == SRN_ACT_SNAKEALT ? launch_t<32, 14, 16, SRN_ACT_SNAKEALT, kPoints, 0, 0>(n, b, pd, ctr, status, s)
                                     : launch_t<32, 14, 16, SRN_ACT_SINE, kPoints, 0, 0>(n, b, pd, ctr, status, s);
  }
  return n.act == SRN_ACT_SNAKEALT ? launch_t<32, 12, 8, SRN_ACT_SNAKEALT, kPoints, 0, 0>(n, b, pd, ctr, status, s)
                                   : launch_t<32, 12, 8, SRN_ACT_SINE, kPoints, 0, 0>(n, b, pd, ctr, status, s);
}

bool density_grad_mma_supported(const NetDev& n) { return render_mma_supported(n, SRN_SHADE_ADJOINT); }

// Density and adjoint input gradient at n points (mode kPointsAdj): the
// forward and backward MMAs of the adjoint-shaded render without the march.
cudaError_t launch_density_grad_mma(const NetDev& n, const float* pts, long long count, float time, float* rho,
                                    float* grad, unsigned long long* ctr, unsigned int* status, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  BatchDev b;
  memset(&b, 0, sizeof(b));
  b.tf.n = 2;
  PointsDev pd{pts, rho, count, time, grad};
  if (n.c == 48) return launch_t<48, 22, 16, SRN_ACT_SNAKEALT, kPointsAdj, 0, 0>(n, b, pd, ctr, status, s);
  if (n.c == 64) return launch_t<64, 30, 16, SRN_ACT_SNAKEALT, kPointsAdj, 0, 0>(n, b, pd, ctr, status, s);
  if (n.m == 14 && n.F == 16)
    return n.act == SRN_ACT_SNAKEALT
               ? launch_t<32, 14, 16, SRN_ACT_SNAKEALT, kPointsAdj, 0, 0>(n, b, pd, ctr, status, s)
               : launch_t<32, 14, 16, SRN_ACT_SINE, kPointsAdj, 0, 0>(n, b, pd, ctr, status, s);
  return n.act == SRN_ACT_SNAKEALT ? launch_t<32, 12, 8, SRN_ACT_SNAKEALT, kPointsAdj, 0, 0>(n, b, pd, ctr, status, s)
                                   : launch_t<32, 12, 8, SRN_ACT_SINE, kPointsAdj, 0, 0>(n, b, pd, ctr, status, s);
}

}  // namespace srn
