// Tensor-core point kernel of the fit (Section 5 world-space training) for
// two-layer networks of width 32 with a density output: forward, loss,
// backward and the layer-0 weight gradient on tcgen05 MMAs; the rest of the
// fit step (cell sort, latent-grid gradient, reductions, Adam) is shared with
// the FP32 path in srn_fit.cu.
//
// A warpgroup takes 128 points at a time, one per thread (thread = MMA row =
// TMEM lane), from a fixed, static assignment of point tiles:
// * forward: the thread writes its layer-0 input row v0 = [sin/cos, p, z, 1, 1]
//   as FP16 blocks [v hi | v lo] (v = hi + lo to ~2^-22); one MMA over the
//   K blocks [v hi | v lo | v hi] (the third re-reads the first) against
//   [W hi | W hi | W lo] (the FP32 master weights split the same way) gives
//   x1 = W0 v0 + b0 in TMEM, FP32-accurate (the bias as FP16 hi + lo weights
//   of the two constant columns);
// * the thread reads x1, applies the activation and its derivative (MUFU
//   sin/cos), evaluates the last layer and the L1 loss in FP32, and forms
//   delta = dL/dx1 = sign(r)/n * w_last * a'(x1);
// * backward to the latent vector: dz = W0_z^T delta in FP32 on the CUDA
//   cores (it feeds the latent-grid gradient, a sum with strong
//   cancellation, so it keeps FP32 accuracy), overlapping the MMA below;
// * weight gradient of layer 0: dW0^T = sum over points of v0 delta^T is an
//   MMA with K = points.  Both operands are read MN-major (one 128-byte row
//   per point): A is the input tile itself (its v hi and v lo blocks, M =
//   128 features), B a tile of the points' delta rows (hi, lo; N = 64), which
//   every thread writes with vector stores.  One MMA per tile accumulates
//   all four hi/lo products in TMEM across the warpgroup's tiles.  The bias
//   gradient of layer 0 is the row of the constant-1 column.  The delta rows are
//   written times 2^s, 2^s >= n (|sign(r)/n| would otherwise fall below the
//   FP16 normal range, 6.1e-5, for n > ~1e4 and lose its hi + lo precision);
//   the accumulated rows are scaled back by 2^-s, exactly.
// * last-layer gradients and the loss are warp reductions in a fixed order.
// Each warpgroup writes one partial row [W | b | loss], reduced in a fixed
// order by the same kernel as the FP32 path's rows: the step is deterministic.
#include "srn_fit.h"
#include "srn_mma_kernel.cuh"
#include "srn_net32.cuh"
#include "srn_sample.cuh"

namespace srn {
namespace {

using namespace mma;

constexpr int kFitWGS = 3;              // warpgroups per CTA (registers: 168 per thread)
constexpr int kFitTmemCols = 512;       // 128 columns per warpgroup (64 forward + 64 dW0), power of two
constexpr int kFitWgCols = 128;

struct FitPlan {
  int oAf, oBt, oB0, oWz, oWl, oFm, oSlot, oMbar, oMisc, total;
};

FitPlan fit_plan(int m, int F) {
  FitPlan p;
  int o = 0;
  p.oAf = o; o += kFitWGS * 2 * kTile;          // input rows [hi | lo] (128 points x 128 FP16)
  p.oBt = o; o += kFitWGS * kTile;              // delta rows [hi | lo] (128 points x 64 FP16)
  p.oB0 = o; o += 3 * 32 * 128;                 // [W hi | W hi | W lo]: 32 rows x 192 columns
  p.oWz = o; o += F * 32 * 4;                    // FP32 latent columns of W0, [F][32]
  p.oWl = o; o += 64 * 4;
  p.oFm = o; o += ((3 * m + 3) & ~3) * 4 + 16;
  p.oSlot = o; o += kFitWGS * 4 * 34 * 4;       // per warp: dW_last[32], db_last, spare
  o = (o + 7) & ~7;
  p.oMbar = o; o += 8 * kFitWGS;
  p.oMisc = o; o += 16 * 4;
  p.total = o + 1024;
  return p;
}

__device__ __forceinline__ uint32_t h16(float v) {
  const __half h = __float2half_rn(v);
  return (uint32_t)__half_as_ushort(h);
}

// MN-major shared-memory descriptor, 128-byte swizzle: one 128-byte row of
// 64 M (or N) elements per K index, 8-row groups 1024 bytes apart (SBO),
// 64-element M blocks `lbo` bytes apart (LBO).
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;  // descriptor version
  d |= (uint64_t)2u << 61;  // SWIZZLE_128B
  return d;
}

// Weight-gradient MMA: M = 128, N = 64, A and B both MN-major (transpose bits).
constexpr uint32_t kIdescGrad = idesc_n(64) | (1u << 15) | (1u << 16);

template <int M, int F, int ACT>
__global__ void __launch_bounds__(128 * kFitWGS, 1)
    fit_mma_kernel(const NetDev net, const PointArgsMma a, const FitPlan plan, unsigned int* __restrict__ status) {
  constexpr int C = 32;
  constexpr int D0 = 3 + 2 * M + F;
  static_assert(D0 + 2 <= 64, "layer-0 input (with the two bias columns) must fit 64 columns");
  constexpr bool SNAKE = ACT == SRN_ACT_SNAKEALT;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* wl = reinterpret_cast<float*>(sm + plan.oWl);
  float* fm = reinterpret_cast<float*>(sm + plan.oFm);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + plan.oMbar);
  volatile int* misc = reinterpret_cast<volatile int*>(sm + plan.oMisc);  // [0] tmem base, [4+wg] fail

  const int tid = threadIdx.x;
  const int wg = tid >> 7, row = tid & 127, lane = tid & 31, warp = row >> 5;
  uint8_t* Af = sm + plan.oAf + wg * 2 * kTile;
  uint8_t* Bt = sm + plan.oBt + wg * kTile;
  uint8_t* B0 = sm + plan.oB0;
  float* wz = reinterpret_cast<float*>(sm + plan.oWz);
  float* slot = reinterpret_cast<float*>(sm + plan.oSlot) + (wg * 4 + warp) * 34;
  float* ex = reinterpret_cast<float*>(Af);  // after the last tile: exchange rows (64 x 33) + 4 loss words

  // ---- stage the FP32 master weights of layer 0 split into FP16 hi + lo.
  // B0 row o: blocks [W hi | W hi | W lo] of 64 columns in the input tile's
  // order; block 0 also carries the bias hi / lo in columns D0, D0+1.
  for (int r = tid; r < C; r += 128 * kFitWGS) {
    for (int cg = 0; cg < 24; ++cg) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t hh[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = 8 * cg + 2 * e + q;
          const int blk = col >> 6, c = col & 63;
          int src = -1;
          if (c < 2 * M) src = (c & 1) ? 3 + M + (c >> 1) : 3 + (c >> 1);
          else if (c < 2 * M + 3) src = c - 2 * M;
          else if (c < D0) src = c;
          float v = 0.0f;
          if (src >= 0) {
            const float wv = net.W[(size_t)r * D0 + src];
            const float wh = __half2float(__float2half_rn(wv));
            v = blk < 2 ? wh : wv - wh;
          }
          if (blk == 0 && (c == D0 || c == D0 + 1)) {
            const float bias = net.b[r];
            const float bh = __half2float(__float2half_rn(bias));
            v = c == D0 ? bh : bias - bh;
          }
          hh[q] = h16(v);
        }
        w[e] = hh[0] | (hh[1] << 16);
      }
      *reinterpret_cast<uint4*>(B0 + (cg >> 3) * (32 * 128) + sw_off(r, cg & 7)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  for (int i = tid; i < F * C; i += 128 * kFitWGS) {
    const int f = i / C, o = i - f * C;
    wz[i] = net.W[(size_t)o * D0 + 3 + 2 * M + f];
  }
  for (int i = tid; i < C; i += 128 * kFitWGS) wl[i] = net.W[(size_t)C * D0 + i];  // FP32 last layer
  if (tid == 0) wl[C] = net.b[C];
  for (int i = tid; i < 3 * M; i += 128 * kFitWGS) fm[i] = net.fourier[i];
  for (int i = row; i < 4 * 34; i += 128) reinterpret_cast<float*>(sm + plan.oSlot)[wg * 4 * 34 + i] = 0.0f;
  if (row == 0) {
    mbar_init(smem_u32(&mbar[wg]), 1);
    misc[4 + wg] = 0;
  }
  if (tid == 0) {
    // row k of a NeRF matrix (Eq. 2): 2 pi 2^(k div 3) on axis k mod 3, zero elsewhere
    int ok = 1;
    for (int k = 0; k < M && ok; ++k)
      for (int ax = 0; ax < 3; ++ax) {
        const float want = (ax == k % 3) ? 6.2831855f * (float)(1 << (k / 3)) : 0.0f;
        if (net.fourier[3 * k + ax] != want) ok = 0;
      }
    misc[2] = ok;
  }
  if (tid < 32) {
    tmem_alloc(smem_u32((const void*)&misc[0]), kFitTmemCols);
    tmem_relinquish();
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const uint32_t tmem = (uint32_t)misc[0];
  const uint32_t d_acc = tmem + (uint32_t)(wg * kFitWgCols);  // forward accumulator (32 of 64 columns)
  const uint32_t d_dw = d_acc + 64;                           // dW0 accumulator (64 columns)
  const uint32_t t_row = d_acc + ((uint32_t)(warp * 32) << 16);
  const uint32_t t_dw = d_dw + ((uint32_t)(warp * 32) << 16);
  const uint32_t af_addr = smem_u32(Af), bt_addr = smem_u32(Bt);
  const uint32_t b0_addr = smem_u32(B0);
  const uint32_t mb = smem_u32(&mbar[wg]);
  const int bar_id = 1 + wg;
  uint32_t phase = 0;
  bool failed = false;

  const net32::Latent lat = net32::make_latent(net, a.time);
  const bool nerf = misc[2] != 0;
  const int step = a.step_ptr ? *a.step_ptr : a.step;
  const float inv_n = 1.0f / (float)a.n;
  // delta rows of the weight-gradient MMA are staged times 2^dexp >= n
  const int dexp = a.n > 1 ? 32 - __clz(a.n - 1) : 0;
  const float dscale = __int_as_float((127 + dexp) << 23), dunscale = __int_as_float((127 - dexp) << 23);
  const int nchunks = (a.n + 127) / 128;
  const int wg_global = blockIdx.x * kFitWGS + wg, n_wg = gridDim.x * kFitWGS;
  float loss_acc = 0.0f;
  bool first = true;

  for (int chunk = wg_global; chunk < nchunks; chunk += n_wg) {
    const int j = chunk * 128 + row;
    const bool valid = j < a.n;
    float3 p = make_float3(0.5f, 0.5f, 0.5f);
    if (valid) p = sample::fit_point(a.cdf, a.cdf_res, a.seed, step, j, a.n);
    // ground truth y = V(p) (trilinear): the eight corner loads issue here,
    // the combination waits until after the forward MMA; the latent corners
    // are gathered first as well, so both latencies overlap the Fourier features
    float yc[8], yfx, yfy, yfz;
    {
      int ix, iy, iz;
      cell_coord(p.x, a.vol.nx, ix, yfx);
      cell_coord(p.y, a.vol.ny, iy, yfy);
      cell_coord(p.z, a.vol.nz, iz, yfz);
      const size_t sy = (size_t)a.vol.nx, sz = (size_t)a.vol.nx * a.vol.ny;
      const float* b = a.vol.vol + iz * sz + iy * sy + ix;
      yc[0] = __ldg(b); yc[1] = __ldg(b + 1); yc[2] = __ldg(b + sy); yc[3] = __ldg(b + sy + 1);
      yc[4] = __ldg(b + sz); yc[5] = __ldg(b + sz + 1); yc[6] = __ldg(b + sz + sy); yc[7] = __ldg(b + sz + sy + 1);
    }

    // ---- layer-0 input v0 in the tile's column order, FP16 hi + lo
    float v[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) v[c] = 0.0f;
    {
      const net32::Cell cell = net32::make_cell(lat, p);
#pragma unroll
      for (int f = 0; f < F; f += 4) {
        const float4 z = net32::latent4(lat, cell, f);
        v[2 * M + 3 + f] = z.x;
        v[2 * M + 4 + f] = z.y;
        v[2 * M + 5 + f] = z.z;
        v[2 * M + 6 + f] = z.w;
      }
    }
    if (nerf) {
      // NeRF rows: one MUFU sin/cos per axis from the argument reduced
      // exactly (x - round(x) in FP32; 2 pi x = w (x - r) + (w - 2 pi) r modulo
      // 2 pi with w the FP32 value of 2 pi), then angle doubling per octave:
      // sin 2t = 2 s c, cos 2t = (c - s)(c + s).  With at most five octaves
      // the doubled error stays below ~2^-17, inside the fit's FP16 hi + lo
      // operand budget.
      static_assert(M <= 15, "at most five octaves without re-seeding");
      float sa[3], ca[3];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int ax = k % 3;
        if (k < 3) {
          const float pa = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
          const float r = rintf(pa);
          __sincosf(fmaf(6.28318548202514648f, pa - r, 1.74845560252379070e-7f * r), &sa[ax], &ca[ax]);
        } else {
          const float ss = sa[ax], cc = ca[ax];
          sa[ax] = 2.0f * ss * cc;
          ca[ax] = (cc - ss) * (cc + ss);
        }
        v[2 * k] = sa[ax];
        v[2 * k + 1] = ca[ax];
      }
    } else {
#pragma unroll
      for (int k = 0; k < M; ++k) {
        float s, c;
        net32::fourier_sincos(fm + 3 * k, p, s, c);
        v[2 * k] = s;
        v[2 * k + 1] = c;
      }
    }
    v[2 * M] = p.x;
    v[2 * M + 1] = p.y;
    v[2 * M + 2] = p.z;
    v[D0] = 1.0f;
    v[D0 + 1] = 1.0f;
#pragma unroll
    for (int cg = 0; cg < 8; ++cg) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        split_h2(v[8 * cg + 2 * e], v[8 * cg + 2 * e + 1], hi[e], lo[e]);
      }
      *reinterpret_cast<uint4*>(Af + sw_tile_off(row, cg)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(Af + sw_tile_off(row, 8 + cg)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    fence_proxy_async();
    tc_fence_before();
    bar_sync(bar_id, 128);
    if (misc[4 + wg]) break;
    if (row == 0 && !a.stall_test) {  // stall_test: no MMA, no commit, nothing in flight
      tc_fence_after();
      // K blocks [v hi | v lo | v hi] x [W hi | W hi | W lo]: the third A block is the first
#pragma unroll
      for (int kk = 0; kk < 12; ++kk) {
        const uint32_t ka = kk >> 2, kb = (kk & 3) * 32;
        mma_f16(d_acc, sw128_desc(af_addr + (ka == 2 ? 0u : ka) * kTile + kb),
                sw128_desc(b0_addr + ka * (32 * 128) + kb), idesc_n(32), kk > 0);
      }
      mma_commit(mb);
    }
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(mb, phase))) {
      failed = true;
      misc[4 + wg] = 1;
    }
    phase ^= 1u;
    tc_fence_after();

    // ---- activation, last layer, loss, delta = dL/dx1
    float x[32];
    if (!failed) tmem_ld32(t_row, x);
    float out = wl[C];
    float dact[32];
#pragma unroll
    for (int o = 0; o < C; ++o) {
      float s, c;
      __sincosf(x[o], &s, &c);
      const float av = SNAKE ? fmaf(0.5f, x[o], s * s) : s;
      dact[o] = SNAKE ? fmaf(2.0f * s, c, 0.5f) : c;
      x[o] = av;  // x now holds the activation
      out = fmaf(wl[o], av, out);
    }
    float y = 0.0f;
    if (valid) {
      const float gx = 1.0f - yfx, gy = 1.0f - yfy, gz = 1.0f - yfz;
      y = gx * gy * gz * yc[0] + yfx * gy * gz * yc[1] + gx * yfy * gz * yc[2] + yfx * yfy * gz * yc[3] +
          gx * gy * yfz * yc[4] + yfx * gy * yfz * yc[5] + gx * yfy * yfz * yc[6] + yfx * yfy * yfz * yc[7];
    }
    const float r = out - y;
    const float dout = valid ? (r > 0.f ? inv_n : (r < 0.f ? -inv_n : 0.f)) : 0.0f;
    if (valid) loss_acc += fabsf(r);
    // last-layer gradients: reduce-scatter dout * a over the warp, lane o keeps output o
    {
      float g[32];
#pragma unroll
      for (int o = 0; o < C; ++o) g[o] = dout * x[o];
#pragma unroll
      for (int w = 16; w > 0; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int o = 0; o < w; ++o) {
          const float send = upper ? g[o] : g[o + w];
          const float keep = upper ? g[o + w] : g[o];
          g[o] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
      }
      slot[lane] += g[0];
      float ds = dout;
#pragma unroll
      for (int w = 16; w > 0; w >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, w);
      if (lane == 0) slot[32] += ds;
    }
    float delta[32];
#pragma unroll
    for (int o = 0; o < C; ++o) delta[o] = dout * wl[o] * dact[o];

    // ---- the point's delta row [hi (32) | lo (32)] (weight gradient, MN-major B)
#pragma unroll
    for (int cg = 0; cg < 4; ++cg) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        split_h2(delta[8 * cg + 2 * e] * dscale, delta[8 * cg + 2 * e + 1] * dscale, hi[e], lo[e]);
      }
      *reinterpret_cast<uint4*>(Bt + sw_off(row, cg)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(Bt + sw_off(row, 4 + cg)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    fence_proxy_async();
    tc_fence_before();
    bar_sync(bar_id, 128);
    if (misc[4 + wg]) break;
    if (row == 0) {
      tc_fence_after();
      // dW0^T += v0^T delta over this tile's points (M = 128: v hi, v lo features; N = 64: delta hi,
      // delta lo; K = 128 points, 16 rows = 2048 bytes per MMA)
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        mma_f16(d_dw, sw128_mn_desc(af_addr + kk * 2048, kTile), sw128_mn_desc(bt_addr + kk * 2048, kTile),
                kIdescGrad, (first && kk == 0) ? 0u : 1u);
      }
      mma_commit(mb);
    }
    first = false;
    // ---- while it runs: latent adjoint dz = W0_z^T delta (FP32), point, cell key
    if (valid) {
      float4* dzj = reinterpret_cast<float4*>(a.dz + (size_t)j * F);
#pragma unroll
      for (int f = 0; f < F; f += 4) {
        float zz[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4* wr = reinterpret_cast<const float4*>(wz + (f + q) * C);
          float acc = 0.0f;
#pragma unroll
          for (int o4 = 0; o4 < C / 4; ++o4) {
            const float4 w4 = wr[o4];
            acc = fmaf(w4.x, delta[4 * o4], acc);
            acc = fmaf(w4.y, delta[4 * o4 + 1], acc);
            acc = fmaf(w4.z, delta[4 * o4 + 2], acc);
            acc = fmaf(w4.w, delta[4 * o4 + 3], acc);
          }
          zz[q] = acc;
        }
        dzj[f >> 2] = make_float4(zz[0], zz[1], zz[2], zz[3]);
      }
      a.pts[3 * (size_t)j] = p.x;
      a.pts[3 * (size_t)j + 1] = p.y;
      a.pts[3 * (size_t)j + 2] = p.z;
      int ix, iy, iz;
      float fx, fy, fz;
      cell_coord(p.x, lat.R, ix, fx);
      cell_coord(p.y, lat.R, iy, fy);
      cell_coord(p.z, lat.R, iz, fz);
      a.key[j] = (unsigned)((iz * (lat.R - 1) + iy) * (lat.R - 1) + ix);
      a.idx[j] = (unsigned)j;
    }
    // the weight-gradient MMA reads this tile's input and delta rows: wait
    // before the next tile overwrites them
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(mb, phase))) {
      failed = true;
      misc[4 + wg] = 1;
    }
    phase ^= 1u;
    tc_fence_after();
  }

  // ---- the warpgroup's partial row [W | b | loss]
  const int nW = C * D0 + C, n_entries = nW + C + 1;
  float* prow = a.part + (size_t)wg_global * (n_entries + 1);
  const bool any_tile = wg_global < nchunks;
  bar_sync(bar_id, 128);
  if (!failed && !misc[4 + wg]) {
    // dW0^T rows: lane f of warps 0-1 holds v0-hi feature f, warps 2-3 the lo
    // feature f - 64; columns: delta hi (0..31), delta lo (32..63)
    float h0[32], h1[32];
    if (any_tile) {
      tmem_ld32(t_dw, h0);
      tmem_ld32(t_dw + 32, h1);
    } else {
#pragma unroll
      for (int o = 0; o < 32; ++o) h0[o] = h1[o] = 0.0f;
    }
#pragma unroll
    for (int o = 0; o < 32; ++o) h0[o] += h1[o];
    if (row >= 64) {
#pragma unroll
      for (int o = 0; o < 32; ++o) ex[(row - 64) * 33 + o] = h0[o];
    }
    bar_sync(bar_id, 128);
    if (row < 64) {
      const int f = row;
      int src = -1;
      if (f < 2 * M) src = (f & 1) ? 3 + M + (f >> 1) : 3 + (f >> 1);
      else if (f < 2 * M + 3) src = f - 2 * M;
      else if (f < D0) src = f;
#pragma unroll
      for (int o = 0; o < 32; ++o) {
        const float g = (h0[o] + ex[f * 33 + o]) * dunscale;  // the delta rows carried 2^dexp
        if (src >= 0) prow[o * D0 + src] = g;
        if (f == D0) prow[nW + o] = g;  // the constant-1 column: bias of layer 0
      }
    }
    // last layer and loss: the four warps' slots in order
    if (row < 32) {
      const float* s0 = reinterpret_cast<float*>(sm + plan.oSlot) + wg * 4 * 34;
      prow[C * D0 + row] = ((s0[row] + s0[34 + row]) + s0[68 + row]) + s0[102 + row];
      if (row == 0) prow[nW + C] = ((s0[32] + s0[66]) + s0[100]) + s0[134];
    }
    // loss: fixed tree over the warpgroup's threads
    float l = loss_acc;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) l += __shfl_xor_sync(0xffffffffu, l, w);
    if (lane == 0) ex[64 * 33 + warp] = l;  // words past the exchange rows
    bar_sync(bar_id, 128);
    if (row == 0) {
      const float* q = ex + 64 * 33;
      prow[n_entries] = ((q[0] + q[1]) + q[2]) + q[3];
    }
  }
  if (failed || misc[4 + wg]) {
    if (row == 0) {
      atomicExch(status, (unsigned int)SRN_ERR_TIMEOUT);
      atomicOr(a.flag, 2u);  // the step's Adam leaves the parameters as they are
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(tmem, kFitTmemCols);
}

template <int M, int F, int ACT>
cudaError_t fit_mma_t(const NetDev& net, const PointArgsMma& a, int grid, unsigned int* status, cudaStream_t st) {
  const FitPlan plan = fit_plan(M, F);
  auto k = fit_mma_kernel<M, F, ACT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.total);
  if (e != cudaSuccess) return e;
  k<<<grid, 128 * kFitWGS, plan.total, st>>>(net, a, plan, status);
  return cudaGetLastError();
}

}  // namespace

int fit_mma_rows_per_cta() { return kFitWGS; }

bool fit_mma_supported(const NetDev& n) {
  if (n.c != 32 || n.l != 2 || n.D != 1 || n.ti) return false;
  if (n.act != SRN_ACT_SINE && n.act != SRN_ACT_SNAKEALT) return false;
  return (n.m == 12 && n.F == 8) || (n.m == 14 && n.F == 16);
}

cudaError_t launch_fit_mma(const NetDev& n, const PointArgsMma& a, int grid, unsigned int* status, cudaStream_t st) {
  if (n.m == 12 && n.F == 8)
    return n.act == SRN_ACT_SNAKEALT ? fit_mma_t<12, 8, SRN_ACT_SNAKEALT>(n, a, grid, status, st)
                                     : fit_mma_t<12, 8, SRN_ACT_SINE>(n, a, grid, status, st);
  return n.act == SRN_ACT_SNAKEALT ? fit_mma_t<14, 16, SRN_ACT_SNAKEALT>(n, a, grid, status, st)
                                   : fit_mma_t<14, 16, SRN_ACT_SINE>(n, a, grid, status, st);
}

}  // namespace srn
