// FP16 tensor-core fV-SRN render for sm_103a: tcgen05.mma with TMEM
// accumulators, persistent CTAs, one thread per ray.
//
// Design (GB300-first restatement of the fused TensorCore network of
// Section 4.1):
// * A CTA holds 7 (6 with finite-difference shading), 4 or 3 warpgroups for
//   hidden width 32, 48 or 64 (what shared memory and registers allow).  Each
//   warpgroup owns a tile of 128 rays, one per thread; thread i of the warpgroup is row i of the MMA operand A and
//   TMEM lane i of the accumulator, so the per-ray work (ray stepping,
//   latent-grid trilinear fetch, Fourier features, transfer function,
//   compositing, early termination) stays one thread per ray as in the paper,
//   while the layers run as M=128 x N=C tensor-core MMAs.
// * Every sample: the thread writes its FP16 layer-0 input row into a
//   K-major shared-memory tile (no swizzle, see a_off); one elected thread
//   issues tcgen05.mma
//   (kind::f16, FP32 accumulate in TMEM); the thread reads its row back with
//   tcgen05.ld, applies the activation in FP32 and writes it into the same
//   tile as the next layer's A row as an FP16 hi + lo pair (a = hi + lo to
//   ~2^-22 relative; the B tile holds [W | W]), so the hidden activations
//   keep FP32 accuracy through the FP16 tensor cores.  Inside the tile the input columns are
//   [sin_0, cos_0, ..., sin_{m-1}, cos_{m-1}, p, z, 1, 1]; the B tile of
//   layer 0 is permuted to match, so the arithmetic is that of [p, sin, cos,
//   z].  Biases ride in the MMA as an FP16 hi + lo pair against two
//   constant-1 columns (layer 0: columns of its own row; hidden layers: one
//   extra K=16 MMA against a constant tile), which keeps them FP32-exact.  The last layer
//   (C -> D) runs on the CUDA cores in FP32.
// * SnakeAlt(x) = 0.5 x + sin^2 x = (x - cos 2x + 1) / 2 (Eq. 3).  Every MMA
//   layer is staged to produce u = 2x (weights and bias doubled, which is
//   exact in FP16), the epilogue hands a = u / 2 - cos u = 2 SnakeAlt(x) - 1
//   to the next layer, and the factor 1/2 and the shift 1/2 are folded into
//   that layer's weights and bias: the doubled next layer then simply uses W
//   and 2b + sum_j W_j.
// * Rays are claimed dynamically from a work counter, a warp at a time: when
//   every lane's ray has terminated (box exit or opacity >= threshold), the
//   warp takes the next 8 x 4 pixel tile.  The lanes then march neighbouring
//   rays in step, so their latent-grid gathers mostly hit the same cells and
//   the L1 serves a warp's loads in few wavefronts (per-lane refill, which
//   keeps every lane busy but scatters the lanes over the volume, was 10 %
//   slower on the config-2 frame).
// * Every mbarrier wait is bounded; on timeout the warpgroup stops, records
//   SRN_ERR_TIMEOUT in the status word and the CTA frees its TMEM.
// * A non-finite network output (an input or activation beyond the FP16
//   range, 65504) is recorded as SRN_ERR_NONFINITE.
#pragma once
#include <string.h>

#include "srn_device.cuh"
#include "srn_mma.h"

namespace srn {
namespace mma {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity) {
  if (mbar_try_wait(a, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(a, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool bar_red_or(int id, int n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, p;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (FP16 inputs, FP32 accumulate).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// Thread's TMEM lane, 32 consecutive FP32 columns, waited for.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (SBO), sm100 descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1u << 46;              // descriptor version
  d |= (uint64_t)2u << 61;              // SWIZZLE_128B
  return d;
}

// Instruction descriptor: kind::f16, A = B = FP16, D = FP32, both K-major,
// M = 128, N = the layer's output width.
constexpr uint32_t idesc_n(int N) { return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24); }

// Byte offset of 16-byte chunk j of row r in a 128B-swizzled tile.
__device__ __forceinline__ uint32_t sw_off(int r, int j) { return (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4)); }

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// FP16 hi + lo split of a pair: hi = fp16(a), lo = fp16(a - hi).  The
// residual a - hi is exact in FP32; it is formed by one mixed-precision FMA
// per element (hi in FP16 times the FP16 constant -1, plus a in FP32), so
// neither widening nor negating hi costs an instruction.
__device__ __forceinline__ void split_h2(float a0, float a1, uint32_t& hi, uint32_t& lo) {
  hi = pack_h2(a0, a1);
  float r0, r1;
  asm("{.reg .b16 x, y, m;\n\t"
      "mov.b32 {x, y}, %2;\n\t"
      "mov.b16 m, 0xBC00;\n\t"
      "fma.rn.f32.f16 %0, x, m, %3;\n\t"
      "fma.rn.f32.f16 %1, y, m, %4;}"
      : "=f"(r0), "=f"(r1)
      : "r"(hi), "f"(a0), "f"(a1));
  lo = pack_h2(r0, r1);
}

// Activation value handed to the next layer from the accumulator value: sin(x)
// for the sine network; for SnakeAlt the accumulator holds u = 2x and the
// value is u / 2 - cos u = 2 SnakeAlt(x) - 1.
template <int ACT>
__device__ __forceinline__ float act_fold(float acc) {
  return ACT == SRN_ACT_SNAKEALT ? fmaf(0.5f, acc, -__cosf(acc)) : __sinf(acc);
}

// Byte offset of 16-byte chunk cg (= column / 8) of row r in a tile of
// 128B-swizzled 128-row K-atoms (the fit kernel's operand tiles).
__device__ __forceinline__ uint32_t sw_tile_off(int r, int cg) {
  return (uint32_t)((cg >> 3) * kTile) + sw_off(r, cg & 7);
}

// A tiles (the per-ray operand rows: layer inputs, activations, adjoint rows)
// are K-major without swizzle: core matrices of 8 rows x 16 bytes, chunk cg
// (= column / 8) of row r at (r / 8) SBO + 128 cg + 16 (r % 8) with
// SBO = NA 1024 for NA 64-column blocks of K.  A thread's chunk offsets are
// then immediates from its row base (no per-store swizzle arithmetic), and a
// quarter-warp's 16-byte stores of one chunk fill 128 contiguous bytes, free
// of bank conflicts.  The tile is NA kTile bytes, as the swizzled one was.
template <int NA>
__device__ __forceinline__ uint32_t a_off(int r, int cg) {
  return (uint32_t)((r >> 3) * (NA * 1024) + cg * 128 + (r & 7) * 16);
}
// Descriptor of such a tile at saddr: leading byte offset 128 (the next core
// matrix along K), stride byte offset NA 1024 (the next 8-row group), no
// swizzle, sm100 descriptor version 1.  K = 16 per MMA advances saddr by 256.
template <int NA>
__device__ __forceinline__ uint64_t a_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((NA * 1024u) >> 4) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// Transfer function with precomputed reciprocal segment widths (same
// segments and lerp as the shared tf_eval).
__device__ __forceinline__ float4 tf_eval_inv(const TFDev& tf, const float* inv, float rho) {
  const float x = clamp01f(rho);
  const int n = tf.n;
  if (x <= tf.pos[0]) return tf.rgba[0];
  if (x >= tf.pos[n - 1]) return tf.rgba[n - 1];
  int i = 0;
  while (i < n - 2 && x >= tf.pos[i + 1]) ++i;
  const float f = (x - tf.pos[i]) * inv[i];
  const float4 a = tf.rgba[i], b = tf.rgba[i + 1];
  return make_float4(fmaf(f, b.x - a.x, a.x), fmaf(f, b.y - a.y, a.y), fmaf(f, b.z - a.z, a.z),
                     fmaf(f, b.w - a.w, a.w));
}

struct RayLat {
  int g0, g1;     // element offsets of the bracketing keyframe grids (g1 < 0: single grid)
  float w0, w1;   // time weights
  float tin;      // time value (input of the direct time encoding)
};

// Latent vector (Section 4.2 trilinear latent grid; Section 7 time blend)
// from the FP16 grid, accumulated in FP32.  Each corner's weight is rounded
// to FP16 and the products taken by mixed-precision FMAs (FP16 weight times
// FP16 grid value, exact, plus the FP32 sum): one instruction per channel
// and corner instead of a widening and an FMA.  The weight rounding (2^-11
// relative) moves z_c by at most 2^-11 sum_k w_k |G_kc|, about as much as the
// FP16 rounding of z itself for the A tile.
// ST: one latent grid (no keyframes), known at compile time: no time blend.
template <int F, int ST>
__device__ __forceinline__ void latent_h(const __half* __restrict__ G, int R, const RayLat& rl, float3 p,
                                         float (&z)[F]) {
  int ix, iy, iz;
  float fx, fy, fz;
  cell_coord(p.x, R, ix, fx);
  cell_coord(p.y, R, iy, fy);
  cell_coord(p.z, R, iz, fz);
  const int sx = F, sy = R * F, sz = R * R * F;
  const int base = iz * sz + iy * sy + ix * sx;
#pragma unroll
  for (int f = 0; f < F; ++f) z[f] = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dz ? fz : 1.0f - fz);
    const int off = base + dx * sx + dy * sy + dz * sz;
#pragma unroll
    for (int kk = 0; kk < (ST ? 1 : 2); ++kk) {
      const int g = ST ? 0 : (kk ? rl.g1 : rl.g0);
      if (!ST && kk && g < 0) break;
      const __half wh = __float2half_rn(ST ? w : w * (kk ? rl.w1 : rl.w0));
      const uint16_t wb = *reinterpret_cast<const uint16_t*>(&wh);
#pragma unroll
      for (int c = 0; c < F; c += 8) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(G + g + off + c));
        const uint32_t qq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          asm("{.reg .b16 x, y, w;\n\t"
              "mov.b32 {x, y}, %2;\n\t"
              "mov.b16 w, %3;\n\t"
              "fma.rn.f32.f16 %0, x, w, %0;\n\t"
              "fma.rn.f32.f16 %1, y, w, %1;}"
              : "+f"(z[c + 2 * e]), "+f"(z[c + 2 * e + 1])
              : "r"(qq[e]), "h"(wb));
        }
      }
    }
  }
}

// Latent vector from the 8-bit grid (Section 4.2: per-channel codes, value
// lo + step * code).  F = 16 codes of a vertex are one 16-byte load; each
// byte is spliced into the FP16 value 1024 + code and 1152 subtracted in
// FP16, both exact, giving the centred code c - 128.  As in latent_h the
// corner weight is rounded to FP16 and sum_k w_k (c_k - 128) accumulated by
// mixed-precision FMAs; since the weights sum to 1,
// z = (lo + 128 step) + step * sum_k w_k (c_k - 128), with lo + 128 step
// staged per channel in qp[2 f].  The weight rounding moves z by at most
// 2^-11 step sum_k w_k |c_k - 128| (half the channel's range, at most).
template <int F, int ST>
__device__ __forceinline__ void latent_q(const uint8_t* __restrict__ Q, const float* qp, int R, const RayLat& rl,
                                         float3 p, float (&z)[F]) {
  static_assert(F == 16, "one 16-byte load per vertex");
  int ix, iy, iz;
  float fx, fy, fz;
  cell_coord(p.x, R, ix, fx);
  cell_coord(p.y, R, iy, fy);
  cell_coord(p.z, R, iz, fz);
  const int sx = F, sy = R * F, sz = R * R * F;
  const int base = iz * sz + iy * sy + ix * sx;
  const __half2 k1152 = __float2half2_rn(1152.0f);
#pragma unroll
  for (int f = 0; f < F; ++f) z[f] = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dz ? fz : 1.0f - fz);
    const int off = base + dx * sx + dy * sy + dz * sz;
#pragma unroll
    for (int kk = 0; kk < (ST ? 1 : 2); ++kk) {
      const int g = ST ? 0 : (kk ? rl.g1 : rl.g0);
      if (!ST && kk && g < 0) break;
      const __half wh = __float2half_rn(ST ? w : w * (kk ? rl.w1 : rl.w0));
      const uint16_t wb = *reinterpret_cast<const uint16_t*>(&wh);
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(Q + g + off));
      const uint32_t words[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t lo2 = __byte_perm(words[e], 0x64646464u, 0x4140u);
        uint32_t hi2 = __byte_perm(words[e], 0x64646464u, 0x4342u);
        const __half2 a2 = __hsub2(*reinterpret_cast<const __half2*>(&lo2), k1152);
        const __half2 b2 = __hsub2(*reinterpret_cast<const __half2*>(&hi2), k1152);
        const uint32_t au = *reinterpret_cast<const uint32_t*>(&a2), bu = *reinterpret_cast<const uint32_t*>(&b2);
        asm("{.reg .b16 x, y, w;\n\t"
            "mov.b32 {x, y}, %4;\n\t"
            "mov.b16 w, %6;\n\t"
            "fma.rn.f32.f16 %0, x, w, %0;\n\t"
            "fma.rn.f32.f16 %1, y, w, %1;\n\t"
            "mov.b32 {x, y}, %5;\n\t"
            "fma.rn.f32.f16 %2, x, w, %2;\n\t"
            "fma.rn.f32.f16 %3, y, w, %3;}"
            : "+f"(z[4 * e]), "+f"(z[4 * e + 1]), "+f"(z[4 * e + 2]), "+f"(z[4 * e + 3])
            : "r"(au), "r"(bu), "h"(wb));
      }
    }
  }
#pragma unroll
  for (int f = 0; f < F; ++f) z[f] = fmaf(qp[2 * f + 1], z[f], qp[2 * f]);
}

// Layer-0 input row (Eq. 1-2 features, Section 4.2 latent vector, Section 7
// time input when TI) in the tile's column order [sin_0, cos_0, ...,
// sin_{m-1}, cos_{m-1}, p, z, (t), 1, 1, 0...] over the K0 columns layer 0
// reads.  Values are packed to FP16 pairs
// and stored 16 bytes at a time as they are produced.
template <int M, int F, int K0, int TI, int GQ, int NA, int ST>
__device__ __forceinline__ void write_input_row(uint8_t* tile, int row, float3 p, bool nerf, const float* fm,
                                                const __half* G, const uint8_t* Q, const float* qp, int R,
                                                const RayLat& rl) {
  constexpr int D0 = 3 + 2 * M + F + TI;
  static_assert(M >= 3, "the NeRF recurrence needs the three base rows");
  float z[F];
  if constexpr (GQ != 0) latent_q<F, ST>(Q, qp, R, rl, p, z);
  else latent_h<F, ST>(G, R, rl, p, z);
  uint32_t w[4];
  int nw = 0, chunk = 0;
  auto emit = [&](float a, float b) {
    w[nw++] = pack_h2(a, b);
    if (nw == 4) {
      *reinterpret_cast<uint4*>(tile + a_off<NA>(row, chunk)) = make_uint4(w[0], w[1], w[2], w[3]);
      ++chunk;
      nw = 0;
    }
  };
  if (nerf) {
    // NeRF rows are 2^j w along axis k mod 3 (octave j = k div 3, w the
    // stored FP32 value of 2 pi): one sin/cos per axis, then angle doubling
    // sin 2t = 2 s c, cos 2t = 1 - 2 s^2 (three instructions; the FMA form's
    // absolute error, about 2^-23, is far below the FP16 rounding of the
    // features for the A tile, 2^-12).  Doubling doubles the error of
    // the base angle, so with more than five octaves the base is recomputed
    // every fourth octave from the reduced argument: with x = 2^j p_a and
    // r = round(x) (both exact in FP32), 2^j w p_a = w (x - r) + (w - 2 pi) r
    // modulo 2 pi.
    constexpr int kReseed = M > 15 ? 4 : 64;
    constexpr float kW = 6.28318548202514648f;         // FP32 2 pi
    constexpr float kWErr = 1.74845560252379070e-7f;    // FP32 2 pi - 2 pi
    float s[3], c[3];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int a = k % 3, j = k / 3;
      const float pa = a == 0 ? p.x : (a == 1 ? p.y : p.z);
      if (j % kReseed == 0) {
        const float x = pa * (float)(1 << j);
        const float r = rintf(x);
        __sincosf(fmaf(kW, x - r, kWErr * r), &s[a], &c[a]);
      } else {
        const float ss = s[a], cc = c[a], t2 = ss + ss;
        s[a] = t2 * cc;
        c[a] = fmaf(-t2, ss, 1.0f);
      }
      emit(s[a], c[a]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const float e = fm[3 * k] * p.x + fm[3 * k + 1] * p.y + fm[3 * k + 2] * p.z;
      float sv, cv;
      sincosf(e, &sv, &cv);
      emit(sv, cv);
    }
  }
  // remaining columns 2M .. K0-1: p, z, the two bias ones, zeros
  float tail[K0 - 2 * M];
#pragma unroll
  for (int i = 0; i < K0 - 2 * M; ++i) {
    const int col = 2 * M + i;
    float v = 0.0f;
    if (col < 2 * M + 3) v = col == 2 * M ? p.x : (col == 2 * M + 1 ? p.y : p.z);
    else if (col < 2 * M + 3 + F) v = z[col - 2 * M - 3];
    else if (col < D0) v = rl.tin;  // Section 7 "direct" time input
    else if (col == D0 || col == D0 + 1) v = 1.0f;
    tail[i] = v;
  }
#pragma unroll
  for (int i = 0; i < K0 - 2 * M; i += 2) emit(tail[i], tail[i + 1]);
}

// ---------------------------------------------------------------- kernel
// Thread's TMEM lane, 16 consecutive FP32 columns, waited for.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Thread's TMEM lane, C consecutive FP32 columns (C a multiple of 16).
template <int C>
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, float (&v)[C]) {
#pragma unroll
  for (int c = 0; c + 32 <= C; c += 32) tmem_ld32(taddr + c, *reinterpret_cast<float(*)[32]>(v + c));
  if constexpr (C % 32 != 0) tmem_ld16(taddr + (C - 16), v + (C - 16));
}

// Thread's TMEM lane, 32 consecutive FP32 columns written, store waited for.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n\t"
      "tcgen05.wait::st.sync.aligned;"
      ::"r"(taddr), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
        "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]),
        "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]),
        "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}

// Thread's TMEM lane, 16 consecutive FP32 columns written, store waited for.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n\t"
      "tcgen05.wait::st.sync.aligned;"
      ::"r"(taddr), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
        "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}

// Thread's TMEM lane, C consecutive FP32 columns written (C a multiple of 16).
template <int C>
__device__ __forceinline__ void tmem_st_row(uint32_t taddr, const float (&v)[C]) {
#pragma unroll
  for (int c = 0; c + 32 <= C; c += 32) tmem_st32(taddr + c, *reinterpret_cast<const float(*)[32]>(v + c));
  if constexpr (C % 32 != 0) tmem_st16(taddr + (C - 16), v + (C - 16));
}

// Gradient with respect to p of sum_c gz[c] z_c(p), z the latent vector
// (trilinear in p inside the cell chosen by cell_coord, time-blended):
// sum over corners and keyframes of w_time (gz . g_corner) grad w_corner(p),
// with d f / d p = R - 1 per axis.
template <int F>
__device__ __forceinline__ float3 latent_grad_h(const __half* __restrict__ G, int R, const RayLat& rl, float3 p,
                                                const float* gz) {
  int ix, iy, iz;
  float fx, fy, fz;
  cell_coord(p.x, R, ix, fx);
  cell_coord(p.y, R, iy, fy);
  cell_coord(p.z, R, iz, fz);
  const int sx = F, sy = R * F, sz = R * R * F;
  const int base = iz * sz + iy * sy + ix * sx;
  float3 g = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const float wx = dx ? fx : 1.0f - fx, wy = dy ? fy : 1.0f - fy, wz = dz ? fz : 1.0f - fz;
    const int off = base + dx * sx + dy * sy + dz * sz;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int gb = kk ? rl.g1 : rl.g0;
      if (kk && gb < 0) break;
      float dot = 0.0f;
#pragma unroll
      for (int c = 0; c < F; c += 8) {
        uint4 q = __ldg(reinterpret_cast<const uint4*>(G + gb + off + c));
        const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 v = __half22float2(h[e]);
          dot = fmaf(gz[c + 2 * e], v.x, dot);
          dot = fmaf(gz[c + 2 * e + 1], v.y, dot);
        }
      }
      dot *= kk ? rl.w1 : rl.w0;
      g.x = fmaf(dot, (dx ? wy : -wy) * wz, g.x);
      g.y = fmaf(dot, wx * (dy ? wz : -wz), g.y);
      g.z = fmaf(dot, wx * (dz ? wy : -wy), g.z);
    }
  }
  const float s = (float)(R - 1);
  return make_float3(s * g.x, s * g.y, s * g.z);
}

template <int C, int M, int F, int ACT, int SH, int TI, int GQ, int LF, int ST>
__global__ void __launch_bounds__(128 * wgs_for(C, SH), 1)
    render_mma_kernel(const NetDev net, const BatchDev b, const PointsDev pd, const SmemPlan plan,
                      unsigned long long* __restrict__ ray_counter, unsigned int* __restrict__ status) {
  constexpr int WGS = wgs_for(C, SH), THREADS = 128 * WGS;
  constexpr int D0 = 3 + 2 * M + F + TI;
  constexpr int K0 = ((D0 + 2 + 15) / 16) * 16;  // inputs + two bias columns
  constexpr int NA0 = (K0 + 63) / 64, NAH = (2 * C + 63) / 64;
  constexpr int BT = C * 128;                    // bytes of one K-atom of a B tile (C rows)
  constexpr uint32_t IDESC = idesc_n(C);
  static_assert(C % 16 == 0 && C <= 64 && K0 <= 128, "shape outside the kernel's tiling");
  constexpr int NP = SH == SRN_SHADE_FD ? 7 : 1;  // network passes per sample
  constexpr bool POINTS = is_points(SH);
  constexpr bool SNAKE = ACT == SRN_ACT_SNAKEALT;
  constexpr bool ADJ = is_adjoint(SH);  // input gradient by backward MMAs (Section 5 "adjoint")
  constexpr int TMC = tmem_cols_for(SH);
  constexpr int NACC = adj_acc_cols(C, K0);  // adjoint: accumulator columns before the derivative stash
  static_assert(!ADJ || (TI == 0 && GQ == 0), "tensor-core adjoint: no time input, FP16 grid");
  static_assert(!ADJ || WGS * tmem_wg_cols(C, SH, K0) <= TMC, "adjoint TMEM layout exceeds the allocation");

  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* Aall = sm + plan.oA;
  uint8_t* B0 = sm + plan.oB0;
  uint8_t* Bh = sm + plan.oBh;
  uint8_t* Bb = sm + plan.oBb;
  uint8_t* BhT = sm + plan.oBhT;
  uint8_t* B0T = sm + plan.oB0T;
  float* wl = reinterpret_cast<float*>(sm + plan.oWl);
  TFDev& tf = *reinterpret_cast<TFDev*>(sm + plan.oTF);
  float* tfinv = reinterpret_cast<float*>(sm + plan.oTFinv);
  float* fm = reinterpret_cast<float*>(sm + plan.oFm);
  float* qp = reinterpret_cast<float*>(sm + plan.oQp);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + plan.oMbar);
  volatile int* misc = reinterpret_cast<volatile int*>(sm + plan.oMisc);  // [0] tmem base, [1] nerf, [4+wg] fail

  const int tid = threadIdx.x;
  const int wg = tid >> 7, row = tid & 127, lane = tid & 31;
  // LF > 0: a network of LF layers and D = 1 output (4 for the gradient
  // head), both fixed at compile time (the layer loop unrolls, the output
  // loop has its exact trip count); the dispatch picks such an instantiation
  // only for such a network
  constexpr int DF = SH == SRN_SHADE_HEAD ? 4 : 1;
  const int L = LF > 0 ? LF : net.l;
  const int D = LF > 0 ? DF : net.D;
  constexpr int NA = NA0 > NAH ? NA0 : NAH;
  // the FP16 latent grid holds G 2^-gexp: the latent columns' layer-0 weights
  // are staged times 2^gexp (exact), the 8-bit grid's lo / step times 2^-gexp
  const int gexp = net.grid_exp ? *net.grid_exp : 0;
  const float gscale = __int_as_float((127 + gexp) << 23);  // 2^gexp, gexp <= 113

  // ---- stage parameters as FP16 B tiles (row o = output neuron, K-major,
  // 128B-swizzled K-atoms).  Layer 0: columns in the tile's input order, FP32
  // bias as hi + lo at D0, D0+1.  Hidden layer h: [W | W] over 2C columns
  // (hi and lo halves of the activation); its bias hi, lo in columns
  // 16(h-1), 16(h-1)+1 of the bias tile (multiplied by the constant tile).
  // SnakeAlt folding as described at the top of the file.  One thread stages
  // one row of one layer.
  for (int it = tid; it < (L - 1) * C; it += THREADS) {
    const int layer = it / C, o = it - layer * C;
    const int din = layer == 0 ? D0 : C;
    const __half* Wsrc = net.W_h + (layer == 0 ? 0 : (size_t)C * D0 + (size_t)(layer - 1) * C * C) + (size_t)o * din;
    float bias = net.b[layer * C + o];
    float scale = 1.0f;
    if (SNAKE) {
      scale = layer == 0 ? 2.0f : 1.0f;
      if (layer > 0) {
        float rs = 0.0f;
        for (int c = 0; c < C; ++c) rs += __half2float(Wsrc[c]);
        bias = 2.0f * bias + rs;
      } else {
        bias = 2.0f * bias;
      }
    }
    const __half bh = __float2half_rn(bias);
    const __half bl = __float2half_rn(bias - __half2float(bh));
    const int ncol = layer == 0 ? K0 : 2 * C;
    uint8_t* Wt = layer == 0 ? B0 : Bh + (layer - 1) * NAH * BT;
    for (int cg = 0; cg < ncol / 8; ++cg) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __half h2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = 8 * cg + 2 * e + q;
          __half v = __float2half_rn(0.0f);
          if (layer == 0) {
            int src = -1;
            if (col < 2 * M) src = (col & 1) ? 3 + M + (col >> 1) : 3 + (col >> 1);
            else if (col < 2 * M + 3) src = col - 2 * M;
            else if (col < D0) src = col;
            const bool lat = src >= 3 + 2 * M && src < 3 + 2 * M + F;
            if (src >= 0) v = __float2half_rn(ldexpf(scale * __half2float(Wsrc[src]), lat ? gexp : 0));
            if (col == D0) v = bh;
            if (col == D0 + 1) v = bl;
          } else {
            v = __float2half_rn(scale * __half2float(Wsrc[col % C]));
          }
          h2[q] = v;
        }
        __half2 hh = __halves2half2(h2[0], h2[1]);
        w[e] = *reinterpret_cast<uint32_t*>(&hh);
      }
      *reinterpret_cast<uint4*>(Wt + (cg >> 3) * BT + sw_off(o, cg & 7)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (layer > 0) {
      const int cg = 2 * (layer - 1);  // the layer's 16-column K-block: chunks cg, cg + 1
      __half2 hb = __halves2half2(bh, bl);
      const uint32_t wb = *reinterpret_cast<uint32_t*>(&hb);
      *reinterpret_cast<uint4*>(Bb + (cg >> 3) * BT + sw_off(o, cg & 7)) = make_uint4(wb, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(Bb + ((cg + 1) >> 3) * BT + sw_off(o, (cg + 1) & 7)) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  if constexpr (ADJ) {
    // backward B tiles, unscaled FP16 weights, K = 2C (hi and lo halves of
    // the adjoint row): hidden layer h (1 <= h <= l-2): row n = input n of
    // the layer, column c -> W_h[c mod C][n]; layer 0: row n = tile input
    // column n (same order as the forward tile; zero for the bias columns and
    // the padding), column c -> W_0[c mod C][src(n)].
    const int rows = (L - 2) * C + K0;
    for (int it = tid; it < rows; it += THREADS) {
      const bool in0 = it >= (L - 2) * C;
      const int h = in0 ? 0 : 1 + it / C;
      const int n = in0 ? it - (L - 2) * C : it - (h - 1) * C;
      int src = n;
      if (in0) {
        if (n < 2 * M) src = (n & 1) ? 3 + M + (n >> 1) : 3 + (n >> 1);
        else if (n < 2 * M + 3) src = n - 2 * M;
        else if (n >= D0) src = -1;
      }
      const int din = in0 ? D0 : C;
      const __half* Wsrc = net.W_h + (in0 ? 0 : (size_t)C * D0 + (size_t)(h - 1) * C * C);
      uint8_t* Wt = in0 ? B0T : BhT + (h - 1) * NAH * BT;
      const int atom = in0 ? K0 * 128 : BT;  // bytes of one K-atom of this tile
      for (int cg = 0; cg < 2 * C / 8; ++cg) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c0 = (8 * cg + 2 * e) % C, c1 = (8 * cg + 2 * e + 1) % C;
          const __half v0 = src >= 0 ? Wsrc[(size_t)c0 * din + src] : __float2half_rn(0.0f);
          const __half v1 = src >= 0 ? Wsrc[(size_t)c1 * din + src] : __float2half_rn(0.0f);
          __half2 hh = __halves2half2(v0, v1);
          w[e] = *reinterpret_cast<uint32_t*>(&hh);
        }
        *reinterpret_cast<uint4*>(Wt + (cg >> 3) * atom + sw_off(n, cg & 7)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
  {
    // last layer on the CUDA cores: folded like the hidden layers
    const __half* Wl = net.W_h + (size_t)C * D0 + (size_t)(L - 2) * C * C;
    for (int i = tid; i < D * C; i += THREADS) wl[i] = (SNAKE ? 0.5f : 1.0f) * __half2float(Wl[i]);
    if (tid < D) {
      float bias = net.b[(L - 1) * C + tid];
      if (SNAKE) {
        float rs = 0.0f;
        for (int c = 0; c < C; ++c) rs += __half2float(Wl[tid * C + c]);
        bias += 0.5f * rs;
      }
      wl[D * C + tid] = bias;
    }
    for (int i = tid; i < 3 * M; i += THREADS) fm[i] = net.fourier[i];
    if (GQ)
      for (int i = tid; i < 2 * F; i += THREADS)  // [lo + 128 step, step] per channel (latent_q)
        qp[i] = ldexpf((i & 1) ? net.grid_qp[i] : fmaf(128.0f, net.grid_qp[i + 1], net.grid_qp[i]), -gexp);
  }
  load_tf(tf, b.tf);
  // the thread's A row starts at zero; the constant tile has ones in columns
  // 0 and 1 of every row (the bias MMA of the hidden layers)
  {
    uint8_t* A = Aall + wg * NA * kTile;
    uint8_t* One = sm + plan.oOne;
    for (int cg = 0; cg < NA * 8; ++cg) *reinterpret_cast<uint4*>(A + a_off<NA>(row, cg)) = make_uint4(0, 0, 0, 0);
    if (wg == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<uint4*>(One + sw_off(row, j)) = make_uint4(j == 0 ? pack_h2(1.0f, 1.0f) : 0u, 0u, 0u, 0u);
    }
  }
  if (row == 0) {
    mbar_init(smem_u32(&mbar[wg]), 1);
    misc[4 + wg] = 0;
  }
  if (tid < 32) {
    tmem_alloc(smem_u32((const void*)&misc[0]), TMC);
    tmem_relinquish();
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    // row k of a NeRF matrix: 2 pi 2^(k div 3) on axis k mod 3, zero elsewhere
    int ok = 1;
    for (int k = 0; k < M && ok; ++k)
      for (int a = 0; a < 3; ++a) {
        const float want = (a == k % 3) ? 6.2831855f * (float)(1 << (k / 3)) : 0.0f;
        if (fm[3 * k + a] != want) ok = 0;
      }
    misc[1] = ok;
  }
  for (int i = tid; i < SRN_MAX_TF_POINTS; i += THREADS) {
    const float wdt = i + 1 < tf.n ? tf.pos[i + 1] - tf.pos[i] : 0.0f;
    tfinv[i] = wdt > 0.0f ? 1.0f / wdt : 0.0f;
  }
  __syncthreads();
  const bool nerf = misc[1] != 0;
  const uint32_t tmem = (uint32_t)misc[0];
  const uint32_t d_tmem = tmem + (uint32_t)(wg * tmem_wg_cols(C, SH, K0));
  const uint32_t t_row = d_tmem + ((uint32_t)((row >> 5) * 32) << 16);  // warp's lane quarter
  uint8_t* A = Aall + wg * NA * kTile;
  const uint32_t a_addr = smem_u32(A), b0_addr = smem_u32(B0), bh_addr = smem_u32(Bh), bb_addr = smem_u32(Bb);
  const uint32_t one_addr = smem_u32(sm + plan.oOne);
  const uint32_t bht_addr = smem_u32(BhT), b0t_addr = smem_u32(B0T);
  const uint32_t mb = smem_u32(&mbar[wg]);
  const int bar_id = 1 + wg;

  // ---- ray state
  const int tiles_x = (b.W + 7) / 8, tiles_y = (b.H + 3) / 4;
  const long long tpf = (long long)tiles_x * tiles_y;
  const long long n_rays = POINTS ? pd.n : tpf * 32 * b.n_views * b.n_times;
  const size_t gsz = (size_t)net.R * net.R * net.R * net.F;
  bool active = false, exhausted = false, failed = false;
  bool overflow = false;  // a non-finite network output (FP16 range exceeded)
  long long pix = 0;
  float3 o = make_float3(0.f, 0.f, 0.f), d = o;
  float t0 = 0.f, t1 = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Acc = 0.f;
  int k = 0, pass = 0;
  RayLat rl{0, -1, 1.0f, 0.0f, 0.0f};
  float rho_c = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  float3 ppos = make_float3(0.f, 0.f, 0.f);
  unsigned int ns = 0;
  uint32_t phase = 0;
  if (POINTS) {
    int k0;
    float f;
    time_weights(net, pd.time, k0, f);
    rl.g0 = (int)(k0 * gsz);
    rl.g1 = net.nkey > 1 ? (int)((k0 + 1) * gsz) : -1;
    rl.w0 = net.nkey > 1 ? 1.0f - f : 1.0f;
    rl.w1 = f;
    rl.tin = pd.time;
  }

  while (true) {
    // ---- refill: a warp whose lanes are all done claims the next 32 rays
    // (one 8 x 4 pixel tile), so its lanes march neighbouring rays together
    while (true) {
      const bool need = !__any_sync(0xffffffffu, active) && !exhausted && !failed;
      const unsigned int mask = __ballot_sync(0xffffffffu, need);
      if (mask == 0) break;
      unsigned long long base = 0;
      const int leader = __ffs(mask) - 1;
      if (lane == leader) base = atomicAdd(ray_counter, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const long long r = (long long)base + __popc(mask & ((1u << lane) - 1u));
        if (r >= n_rays) {
          exhausted = true;
        } else if (POINTS) {
          pix = r;
          ppos = make_float3(clamp01f(pd.pts[3 * r]), clamp01f(pd.pts[3 * r + 1]), clamp01f(pd.pts[3 * r + 2]));
          active = true;
        } else {
          const long long tile = r >> 5;
          const int li = (int)(r & 31);
          const long long frame = tile / tpf;
          const int tt = (int)(tile - frame * tpf);
          const int px = (tt % tiles_x) * 8 + (li & 7), py = (tt / tiles_x) * 4 + (li >> 3);
          if (px < b.W && py < b.H) {
            const int view = (int)(frame % b.n_views), ti = (int)(frame / b.n_views);
            pix = (frame * b.H + py) * (long long)b.W + px;
            camera_ray(b.cams[view], b.W, b.H, px, py, o, d);
            if (box_intersect(o, d, t0, t1)) {
              int k0;
              float f;
              time_weights(net, b.times[ti], k0, f);
              rl.g0 = (int)(k0 * gsz);
              rl.g1 = net.nkey > 1 ? (int)((k0 + 1) * gsz) : -1;
              rl.w0 = net.nkey > 1 ? 1.0f - f : 1.0f;
              rl.w1 = f;
              rl.tin = b.times[ti];
              C0 = C1 = C2 = Acc = 0.f;
              k = 0;
              pass = 0;
              active = true;
            } else {
              reinterpret_cast<float4*>(b.out)[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
        }
      }
    }

    // ---- layer-0 input of this pass
    float len = 0.f;
    float3 qs = make_float3(0.f, 0.f, 0.f);  // sample position of this pass
    if (POINTS && active && !failed) {
      write_input_row<M, F, K0, TI, GQ, NA, ST>(A, row, ppos, nerf, fm, net.grid_h, net.grid_q, qp, net.R, rl);
      qs = ppos;
    } else if (active && !failed) {
      const float ta = fmaf((float)k, b.step, t0);
      const float tb = fminf(fmaf((float)(k + 1), b.step, t0), t1);
      len = tb - ta;
      const float tm = 0.5f * (ta + tb);
      float3 q = make_float3(clamp01f(fmaf(tm, d.x, o.x) + 0.5f), clamp01f(fmaf(tm, d.y, o.y) + 0.5f),
                             clamp01f(fmaf(tm, d.z, o.z) + 0.5f));
      if (SH == SRN_SHADE_FD && pass > 0) {
        const int ax = (pass - 1) >> 1;
        const float h = (pass & 1) ? b.fd_h : -b.fd_h;
        if (ax == 0) q.x = clamp01f(q.x + h);
        if (ax == 1) q.y = clamp01f(q.y + h);
        if (ax == 2) q.z = clamp01f(q.z + h);
      }
      write_input_row<M, F, K0, TI, GQ, NA, ST>(A, row, q, nerf, fm, net.grid_h, net.grid_q, qp, net.R, rl);
      qs = q;
    }
    fence_proxy_async();
    tc_fence_before();
    const bool any = bar_red_or(bar_id, 128, active && !failed);
    if (!any || misc[4 + wg]) break;
    if (row == 0 && !b.stall_test) {  // stall_test: no MMA, no commit, nothing in flight
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < K0 / 16; ++kk) {
        const uint32_t ka = ((16 * kk) >> 6), kb = ((16 * kk) & 63) * 2;
        mma_f16(d_tmem, a_desc<NA>(a_addr + kk * 256), sw128_desc(b0_addr + ka * BT + kb), IDESC, kk > 0);
      }
      mma_commit(mb);
    }

    // ---- layers: wait, read the accumulator row, activation, next MMA
    float out[4] = {0.f, 0.f, 0.f, 0.f};
    float dl[C];  // adjoint variant: d out / d (pre-activation) of the current layer
    bool stop = false;
#pragma unroll(LF > 0 ? LF - 1 : 1)
    for (int layer = 0; layer < L - 1; ++layer) {
      // the failure decision is warp-uniform so tcgen05.ld stays convergent;
      // a failed thread keeps arriving at the warpgroup barriers, which all
      // threads leave together once the flag is visible
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(mb, phase))) {
        failed = true;
        misc[4 + wg] = 1;
      }
      phase ^= 1u;
      tc_fence_after();
      float x[C];
      if (!failed) tmem_ld_row<C>(t_row, x);
      if (layer < L - 2) {
        if (!failed) {
          // activation as FP16 hi (columns 0..C-1) + lo (columns C..2C-1)
#pragma unroll
          for (int j = 0; j < C / 8; ++j) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              split_h2(act_fold<ACT>(x[8 * j + 2 * e]), act_fold<ACT>(x[8 * j + 2 * e + 1]), hi[e], lo[e]);
            }
            *reinterpret_cast<uint4*>(A + a_off<NA>(row, j)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(A + a_off<NA>(row, C / 8 + j)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
          if constexpr (ADJ) {
            // activation derivative of this hidden layer, kept in TMEM for the
            // backward: SnakeAlt' = 0.5 + sin(2x) (the accumulator holds 2x); sin' = cos
            float dv[C];
#pragma unroll
            for (int j = 0; j < C; ++j) dv[j] = SNAKE ? 0.5f + __sinf(x[j]) : __cosf(x[j]);
            tmem_st_row<C>(t_row + NACC + C * layer, dv);
          }
        }
        fence_proxy_async();
        tc_fence_before();
        bar_sync(bar_id, 128);
        if (misc[4 + wg]) { stop = true; break; }
        if (row == 0) {
          tc_fence_after();
          const uint32_t bw = bh_addr + layer * NAH * BT;
          const uint32_t kbias = 16 * layer;  // this layer's K-block of the bias tile
          mma_f16(d_tmem, sw128_desc(one_addr), sw128_desc(bb_addr + (kbias >> 6) * BT + (kbias & 63) * 2), IDESC,
                  0u);
#pragma unroll
          for (int kk = 0; kk < 2 * C / 16; ++kk) {
            const uint32_t ka = ((16 * kk) >> 6), kb = ((16 * kk) & 63) * 2;
            mma_f16(d_tmem, a_desc<NA>(a_addr + kk * 256), sw128_desc(bw + ka * BT + kb), IDESC, 1u);
          }
          mma_commit(mb);
        }
      } else if (!failed) {
        float a[C];
#pragma unroll
        for (int j = 0; j < C; ++j) a[j] = act_fold<ACT>(x[j]);
#pragma unroll
        for (int dd = 0; dd < 4; ++dd) {
          if (dd < D) {
            float sacc = wl[D * C + dd];
#pragma unroll
            for (int j = 0; j < C; ++j) sacc = fmaf(wl[dd * C + j], a[j], sacc);
            out[dd] = sacc;
          }
        }
        if constexpr (ADJ) {
          // d out / d x of the last hidden layer; wl holds W / 2 for SnakeAlt
#pragma unroll
          for (int j = 0; j < C; ++j) dl[j] = SNAKE ? wl[j] * fmaf(2.0f, __sinf(x[j]), 1.0f) : wl[j] * __cosf(x[j]);
        }
      }
    }
    if (stop) break;

    // ---- adjoint input gradient (Section 5): backward through the hidden
    // layers and layer 0 on the tensor cores, the adjoint row split into FP16
    // hi + lo like the activations; then the Fourier and latent Jacobians.
    float3 gadj = make_float3(0.f, 0.f, 0.f);
    if constexpr (ADJ) {
      for (int h = L - 2; h >= 0; --h) {
        if (!failed) {
#pragma unroll
          for (int j = 0; j < C / 8; ++j) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              split_h2(dl[8 * j + 2 * e], dl[8 * j + 2 * e + 1], hi[e], lo[e]);
            }
            *reinterpret_cast<uint4*>(A + a_off<NA>(row, j)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(A + a_off<NA>(row, C / 8 + j)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
        fence_proxy_async();
        tc_fence_before();
        bar_sync(bar_id, 128);
        if (misc[4 + wg]) { stop = true; break; }
        if (row == 0) {
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 2 * C / 16; ++kk) {
            const uint32_t ka = ((16 * kk) >> 6), kb = ((16 * kk) & 63) * 2;
            const uint64_t ad = a_desc<NA>(a_addr + kk * 256);
            if (h >= 1)
              mma_f16(d_tmem, ad, sw128_desc(bht_addr + (h - 1) * NAH * BT + ka * BT + kb), IDESC, kk > 0);
            else
              mma_f16(d_tmem, ad, sw128_desc(b0t_addr + ka * (K0 * 128) + kb), idesc_n(K0), kk > 0);
          }
          mma_commit(mb);
        }
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(mb, phase))) {
          failed = true;
          misc[4 + wg] = 1;
        }
        phase ^= 1u;
        tc_fence_after();
        if (failed) continue;
        if (h >= 1) {
          float g[C], dv[C];
          tmem_ld_row<C>(t_row, g);
          tmem_ld_row<C>(t_row + NACC + C * (h - 1), dv);
#pragma unroll
          for (int j = 0; j < C; ++j) dl[j] = g[j] * dv[j];
        } else {
          float gv[K0];
          tmem_ld_row<K0>(t_row, gv);
          if (active) {
            // position columns, then the Fourier features (d sin e = cos e F_k,
            // d cos e = -sin e F_k), then the latent vector
            float3 gp = make_float3(gv[2 * M], gv[2 * M + 1], gv[2 * M + 2]);
            if (nerf) {
              constexpr int kReseed = M > 15 ? 4 : 64;
              constexpr float kW = 6.28318548202514648f, kWErr = 1.74845560252379070e-7f;
              float sn[3], cs[3];
              float ga[3] = {0.f, 0.f, 0.f};
#pragma unroll
              for (int kq = 0; kq < M; ++kq) {
                const int a = kq % 3, j = kq / 3;
                const float pa = a == 0 ? qs.x : (a == 1 ? qs.y : qs.z);
                if (j % kReseed == 0) {
                  const float xx = pa * (float)(1 << j);
                  const float r = rintf(xx);
                  __sincosf(fmaf(kW, xx - r, kWErr * r), &sn[a], &cs[a]);
                } else {
                  const float ss = sn[a], cc = cs[a];
                  sn[a] = 2.0f * ss * cc;
                  cs[a] = (cc - ss) * (cc + ss);
                }
                ga[a] = fmaf(fm[3 * kq + a], gv[2 * kq] * cs[a] - gv[2 * kq + 1] * sn[a], ga[a]);
              }
              gp.x += ga[0];
              gp.y += ga[1];
              gp.z += ga[2];
            } else {
#pragma unroll
              for (int kq = 0; kq < M; ++kq) {
                const float e = fm[3 * kq] * qs.x + fm[3 * kq + 1] * qs.y + fm[3 * kq + 2] * qs.z;
                float sv, cv;
                sincosf(e, &sv, &cv);
                const float coef = gv[2 * kq] * cv - gv[2 * kq + 1] * sv;
                gp.x = fmaf(coef, fm[3 * kq], gp.x);
                gp.y = fmaf(coef, fm[3 * kq + 1], gp.y);
                gp.z = fmaf(coef, fm[3 * kq + 2], gp.z);
              }
            }
            float3 gl = latent_grad_h<F>(net.grid_h, net.R, rl, qs, gv + 2 * M + 3);
            gl = make_float3(gl.x * gscale, gl.y * gscale, gl.z * gscale);  // grid_h = G 2^-gexp
            gadj = make_float3(gp.x + gl.x, gp.y + gl.y, gp.z + gl.z);
          }
        }
      }
      if (stop) break;
    }

    if (POINTS) {
      if (active && !failed) {
        if constexpr (ADJ) {
          // density and gradient mode: out is the density [n] (output 0 of a
          // 4-output head), grad [n][3]
          pd.out[pix] = out[0];
          if (pd.grad) {
            pd.grad[3 * pix] = gadj.x;
            pd.grad[3 * pix + 1] = gadj.y;
            pd.grad[3 * pix + 2] = gadj.z;
          }
        } else {
          for (int dd = 0; dd < D; ++dd) pd.out[pix * D + dd] = out[dd];
        }
        overflow |= !(fabsf(out[0]) < INFINITY);
        ++ns;
        active = false;
      }
      continue;
    }
    // ---- transfer function, shading, compositing, termination
    if (active && !failed) {
      bool sample_done = true;
      float3 g = make_float3(0.f, 0.f, 0.f);
      if (SH == SRN_SHADE_FD) {
        if (pass == 0) rho_c = out[0];
        else if (pass == 1) gx = out[0];
        else if (pass == 2) gx = (gx - out[0]) / (2.0f * b.fd_h);
        else if (pass == 3) gy = out[0];
        else if (pass == 4) gy = (gy - out[0]) / (2.0f * b.fd_h);
        else if (pass == 5) gz = out[0];
        else gz = (gz - out[0]) / (2.0f * b.fd_h);
        sample_done = pass == NP - 1;
        pass = sample_done ? 0 : pass + 1;
        g = make_float3(gx, gy, gz);
      } else {
        rho_c = out[0];
        if (SH == SRN_SHADE_HEAD) g = make_float3(out[1], out[2], out[3]);
        if (ADJ) g = gadj;
      }
      if (sample_done) {
        ++ns;
        overflow |= !(fabsf(rho_c) < INFINITY);
        float4 c = tf_eval_inv(tf, tfinv, rho_c);
        const float alpha = 1.0f - __expf(-c.w * tf.opacity_scale * len);
        if (SH != SRN_SHADE_NONE) shade(c, g, d);
        const float w = (1.0f - Acc) * alpha;
        C0 = fmaf(w, c.x, C0);
        C1 = fmaf(w, c.y, C1);
        C2 = fmaf(w, c.z, C2);
        Acc += w;
        ++k;
        if (Acc >= b.et || fmaf((float)k, b.step, t0) >= t1) {
          reinterpret_cast<float4*>(b.out)[pix] = make_float4(C0, C1, C2, Acc);
          active = false;
        }
      }
    }
  }

  if (failed || misc[4 + wg]) {
    if (row == 0) atomicExch(status, (unsigned int)SRN_ERR_TIMEOUT);
  } else if (__any_sync(0xffffffffu, overflow) && lane == 0) {
    // an input or activation outside the FP16 range made the output
    // non-finite; the FP32 path evaluates such networks
    atomicCAS(status, (unsigned int)SRN_OK, (unsigned int)SRN_ERR_NONFINITE);
  }
  if (!POINTS) add_samples(b.samples, ns);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(tmem, TMC);
}

template <int C, int M, int F, int ACT, int SH, int TI, int GQ, int LF, int ST>
cudaError_t launch_t(const NetDev& net, const BatchDev& b, const PointsDev& pd, unsigned long long* ctr,
                     unsigned int* status, cudaStream_t s) {
  if (LF > 0 && (net.l != LF || net.D != (SH == SRN_SHADE_HEAD ? 4 : 1))) return cudaErrorInvalidValue;
  if (ST && net.nkey != 1) return cudaErrorInvalidValue;
  SmemPlan plan = make_plan(net, C, wgs_for(C, SH), is_adjoint(SH));
  auto k = render_mma_kernel<C, M, F, ACT, SH, TI, GQ, LF, ST>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.total);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k<<<sms, 128 * wgs_for(C, SH), plan.total, s>>>(net, b, pd, plan, ctr, status);
  return cudaGetLastError();
}

// Explicit instantiation of one variant (used by the srn_mma_w*.cu units);
// SRN_MMA_INSTANTIATE_L fixes the layer count (LF) and whether the network
// has a single latent grid (ST).
#define SRN_MMA_INSTANTIATE_L(C, M, F, ACT, SH, TI, GQ, LF, ST)                                                  \
  template cudaError_t launch_t<C, M, F, ACT, SH, TI, GQ, LF, ST>(const NetDev&, const BatchDev&,               \
                                                                  const PointsDev&, unsigned long long*,        \
                                                                  unsigned int*, cudaStream_t);
#define SRN_MMA_INSTANTIATE(C, M, F, ACT, SH, TI, GQ) SRN_MMA_INSTANTIATE_L(C, M, F, ACT, SH, TI, GQ, 0, 0)

}  // namespace mma
}  // namespace srn
