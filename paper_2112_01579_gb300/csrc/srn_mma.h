// Declarations shared by the tensor-core render kernel (srn_mma_kernel.cuh),
// its explicit instantiations (srn_mma_k*.cu) and the dispatcher
// (srn_mma.cu).  Each kernel variant is compiled in exactly one translation
// unit, so the variants build in parallel.
#pragma once
#include "srn_internal.h"

namespace srn {
namespace mma {


constexpr int kPoints = 4;     // kernel mode: network output at given points (no ray march)
constexpr int kPointsAdj = 5;  // kernel mode: density and adjoint input gradient at given points
constexpr bool is_adjoint(int SH) { return SH == SRN_SHADE_ADJOINT || SH == kPointsAdj; }
constexpr bool is_points(int SH) { return SH == kPoints || SH == kPointsAdj; }

// Warpgroups per CTA for hidden width C and shading mode SH (one CTA per
// SM): what the shared memory of the A tiles and weight tiles and the
// register file allow.  Width 32 runs 7 (72 registers a thread), except the
// finite-difference variant, whose extra state needs the 80 registers of 6,
// and the adjoint variants, whose TMEM stash limits them to 4.
constexpr int wgs_for(int C, int SH) {
  return is_adjoint(SH) ? (C == 32 ? 4 : 2)
                        : (C == 32 ? (SH == SRN_SHADE_FD ? 6 : 7) : (C == 48 ? 4 : 3));
}
constexpr int kAdjMaxLayers = 4;  // layers of the networks the tensor-core adjoint takes
// TMEM columns a CTA allocates, and the columns of one warpgroup.  The
// adjoint variants keep an accumulator wide enough for the input-gradient
// MMA (N = K0, the layer-0 input columns) and for the hidden layers (N = C),
// rounded up to 32 columns, followed by the stashed activation derivatives
// of the (at most two) hidden layers, C columns each: 64 + 64 (width 32, four
// warpgroups), 96 + 96 (48, two), 96 + 128 (64, two).
constexpr int tmem_cols_for(int SH) { return is_adjoint(SH) ? 512 : 256; }
constexpr int adj_acc_cols(int C, int K0) { return (((K0 > C ? K0 : C) + 31) / 32) * 32; }
constexpr int tmem_wg_cols(int C, int SH, int K0) {
  return is_adjoint(SH) ? adj_acc_cols(C, K0) + (kAdjMaxLayers - 2) * C : C;
}
constexpr int kTile = 128 * 128;       // 128 rows x 128 B (64 FP16 columns): an A-tile block, the constant tile

constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

// Point-evaluation arguments (modes kPoints, kPointsAdj).
struct PointsDev {
  const float* pts;  // [n][3]
  float* out;        // [n][D] (kPointsAdj: density [n])
  long long n;
  float time;
  float* grad;       // kPointsAdj: d rho / d p [n][3], or null
};

// ---------------------------------------------------------------- layout
struct SmemPlan {
  int oA, oOne, oB0, oBh, oBb, oBhT, oB0T, oWl, oTF, oTFinv, oFm, oQp, oMbar, oMisc, total;
};

// Shared memory for hidden width C and WGS warpgroups.  An operand row spans
// ceil(K / 64) blocks of 64 FP16 columns: a warpgroup's A tile (128 rows,
// unswizzled core-matrix layout, see a_off) takes kTile bytes per block; B
// tiles are 128B-swizzled K-atoms C * 128 bytes apart.
inline SmemPlan make_plan(const NetDev& n, int C, int WGS, bool adjoint = false) {
  const int D0 = net_d0(n);
  const int K0 = ((D0 + 2 + 15) / 16) * 16;
  const int NA0 = (K0 + 63) / 64, NAH = (2 * C + 63) / 64, NA = NA0 > NAH ? NA0 : NAH;
  const int BT = C * 128;
  const int NBB = n.l > 2 ? (16 * (n.l - 2) + 63) / 64 : 1;
  SmemPlan s;
  int o = 0;
  s.oA = o; o += WGS * NA * kTile;
  s.oOne = o; o += kTile;                   // constant tile: columns 0, 1 = 1
  s.oB0 = o; o += NA0 * BT;                 // layer 0
  s.oBh = o; o += (n.l - 2) * NAH * BT;     // hidden layers: [W | W]
  s.oBb = o; o += NBB * BT;                 // hidden biases, one 16-column K-block per layer
  s.oBhT = o; if (adjoint) o += (n.l - 2) * NAH * BT;      // adjoint: [W_h^T | W_h^T] of the hidden layers
  s.oB0T = o; if (adjoint) o += NAH * (NA0 * 64) * 128;    // adjoint: [W_0^T | W_0^T], K0 rows
  s.oWl = o; o += (n.D * C + 4) * 4;
  o = (o + 15) & ~15;
  s.oTF = o; o += (int)sizeof(TFDev);
  o = (o + 15) & ~15;
  s.oTFinv = o; o += SRN_MAX_TF_POINTS * 4;
  s.oFm = o; o += ((3 * n.m + 3) & ~3) * 4 + 16;
  s.oQp = o; o += 2 * 32 * 4;
  o = (o + 7) & ~7;
  s.oMbar = o; o += 8 * WGS;
  s.oMisc = o; o += 16 * 4;
  s.total = o + 1024;  // alignment slack
  return s;
}

// One kernel variant: hidden width C, M Fourier rows, F latent channels,
// activation ACT, shading SH (or kPoints), direct time input TI, 8-bit grid
// GQ; LF > 0: a network of LF layers and D = 1 output (4 with head
// shading), both fixed at compile time (0: read from the network); ST = 1:
// a single latent grid (no keyframes), so the gather has no time blend.
// Defined in srn_mma_kernel.cuh, instantiated in srn_mma_w*.cu.
template <int C, int M, int F, int ACT, int SH, int TI, int GQ, int LF = 0, int ST = 0>
cudaError_t launch_t(const NetDev& net, const BatchDev& b, const PointsDev& pd, unsigned long long* ctr,
                     unsigned int* status, cudaStream_t s);

}  // namespace mma
}  // namespace srn
