// FP32 network device code shared by the render / eval kernels and the fit
// kernels: shared-memory staging of the parameters, the forward pass
// (Section 3 layer equation, Eq. 1-2 Fourier features, Section 4.2 latent
// grid) and the adjoint input gradient (Section 5 "Adjoint").
#pragma once

#include "srn_device.cuh"
#include "srn_df.cuh"

namespace srn {
namespace net32 {

constexpr int kMaxL = 8;  // deepest network the FP32 kernels stash for the adjoint

// Shared-memory image of the network, offsets in floats (multiples of 4).
struct Layout {
  int d0, l, D, m, F, ti;
  int oF, oW0T, ob0, oHid, hidStride, oWl, obl, total;
  int rowmajor;
};

inline Layout make_layout(const NetDev& n, bool rowmajor) {
  Layout L;
  const int C = n.c;
  L.d0 = net_d0(n); L.l = n.l; L.D = n.D; L.m = n.m; L.F = n.F; L.ti = n.ti;
  L.rowmajor = rowmajor ? 1 : 0;
  int o = 0;
  L.oF = o; o += ((3 * n.m + 3) / 4) * 4;
  L.oW0T = o; o += L.d0 * C;
  L.ob0 = o; o += C;
  L.oHid = o; L.hidStride = C * C + C + (rowmajor ? C * C : 0);
  o += (n.l - 2) * L.hidStride;
  L.oWl = o; o += n.D * C;
  L.obl = o; o += 4;
  L.total = o;
  return L;
}

// Stage the FP32 parameters: W0 and hidden layers transposed ([in][out]) so a
// thread adds one input's contribution to all outputs with float4 reads; the
// last layer row-major; hidden layers also row-major for the adjoint.
template <int C>
__device__ void load_net(float* sm, const Layout& L, const NetDev& n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 3 * L.m; i += nt) sm[L.oF + i] = n.fourier[i];
  const float* W = n.W;
  for (int i = tid; i < L.d0 * C; i += nt) {
    int o = i / L.d0, j = i - o * L.d0;
    sm[L.oW0T + j * C + o] = W[i];
  }
  for (int i = tid; i < C; i += nt) sm[L.ob0 + i] = n.b[i];
  W += (size_t)L.d0 * C;
  const float* bb = n.b + C;
  for (int h = 0; h < L.l - 2; ++h) {
    float* base = sm + L.oHid + h * L.hidStride;
    for (int i = tid; i < C * C; i += nt) {
      int o = i / C, j = i - o * C;
      base[j * C + o] = W[i];
      if (L.rowmajor) base[C * C + C + i] = W[i];
    }
    for (int i = tid; i < C; i += nt) base[C * C + i] = bb[i];
    W += C * C;
    bb += C;
  }
  for (int i = tid; i < L.D * C; i += nt) sm[L.oWl + i] = W[i];
  for (int i = tid; i < L.D; i += nt) sm[L.obl + i] = bb[i];
  __syncthreads();
}

// h += a * row, two outputs per packed FP32x2 FMA (each lane a correctly
// rounded FMA, so the same bits as scalar fmaf).
template <int C>
__device__ __forceinline__ void axpy(float (&h)[C], const float* __restrict__ row, float a) {
  const float2 aa = make_float2(a, a);
#pragma unroll
  for (int o = 0; o < C; o += 4) {
    const float4 w = *reinterpret_cast<const float4*>(row + o);
    const float2 r0 = __ffma2_rn(make_float2(w.x, w.y), aa, make_float2(h[o], h[o + 1]));
    const float2 r1 = __ffma2_rn(make_float2(w.z, w.w), aa, make_float2(h[o + 2], h[o + 3]));
    h[o] = r0.x;
    h[o + 1] = r0.y;
    h[o + 2] = r1.x;
    h[o + 3] = r1.y;
  }
}

template <int C>
__device__ __forceinline__ float dotrow(const float* __restrict__ row, const float (&a)[C]) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int o = 0; o < C; o += 4) {
    float4 w = *reinterpret_cast<const float4*>(row + o);
    s0 = fmaf(w.x, a[o], s0);
    s1 = fmaf(w.y, a[o + 1], s1);
    s2 = fmaf(w.z, a[o + 2], s2);
    s3 = fmaf(w.w, a[o + 3], s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// Eq. 3 SnakeAlt(x) = 0.5 x + sin^2 x, or sin(x); and their derivatives.
// Out-of-line sin / cos: the accurate functions carry a large argument-
// reduction path, and inlined once per hidden unit of the unrolled layers
// they overflow the instruction cache (the fit kernel stalled mostly on
// instruction fetch).
static __device__ __noinline__ void sincos_call(float x, float* s, float* c) { sincosf(x, s, c); }
static __device__ __noinline__ float sin_call(float x) { return sinf(x); }

__device__ __forceinline__ float act_f(int act, float x) {
  float s = sin_call(x);
  return act == SRN_ACT_SNAKEALT ? fmaf(0.5f, x, s * s) : s;
}
// Activation value and derivative from one sin/cos evaluation.
__device__ __forceinline__ void act_and_df(int act, float x, float& a, float& d) {
  float s, c;
  sincos_call(x, &s, &c);
  if (act == SRN_ACT_SNAKEALT) {
    a = fmaf(0.5f, x, s * s);
    d = 0.5f + 2.0f * s * c;
  } else {
    a = s;
    d = c;
  }
}
__device__ __forceinline__ float act_df(int act, float x) {
  if (act == SRN_ACT_SNAKEALT) {
    float s, c;
    sincosf(x, &s, &c);
    return 0.5f + 2.0f * s * c;
  }
  return cosf(x);
}

// Latent grid source of one frame: z = tw0 G_k0(p) + tw1 G_k0+1(p).
struct Latent {
  const float* g0;
  const float* g1;
  float tw0, tw1;
  float tin;  // time value (the extra input of the direct time encoding)
  int R, F;
};

__device__ __forceinline__ Latent make_latent(const NetDev& n, float t) {
  int k0;
  float f;
  time_weights(n, t, k0, f);
  size_t gsz = (size_t)n.R * n.R * n.R * n.F;
  Latent L;
  L.g0 = n.grid + (size_t)k0 * gsz;
  L.g1 = n.nkey > 1 ? L.g0 + gsz : nullptr;
  L.tw0 = n.nkey > 1 ? 1.0f - f : 1.0f;
  L.tw1 = f;
  L.tin = t;
  L.R = n.R;
  L.F = n.F;
  return L;
}

struct Cell {
  int base, sx, sy, sz;   // element offsets of vertex (ix,iy,iz) and of +x, +y, +z
  float fx, fy, fz;
};

__device__ __forceinline__ Cell make_cell(const Latent& lat, float3 p) {
  Cell c;
  int ix, iy, iz;
  cell_coord(p.x, lat.R, ix, c.fx);
  cell_coord(p.y, lat.R, iy, c.fy);
  cell_coord(p.z, lat.R, iz, c.fz);
  c.sx = lat.F;
  c.sy = lat.R * lat.F;
  c.sz = lat.R * lat.R * lat.F;
  c.base = iz * c.sz + iy * c.sy + ix * c.sx;
  return c;
}

// Channels f..f+3 of the latent vector (trilinear, time-blended).
__device__ __forceinline__ float4 latent4(const Latent& lat, const Cell& c, int f) {
  float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    float w = (dx ? c.fx : 1.0f - c.fx) * (dy ? c.fy : 1.0f - c.fy) * (dz ? c.fz : 1.0f - c.fz);
    int off = c.base + dx * c.sx + dy * c.sy + dz * c.sz + f;
    float4 g = __ldg(reinterpret_cast<const float4*>(lat.g0 + off));
    float w0 = w * lat.tw0;
    z.x = fmaf(w0, g.x, z.x); z.y = fmaf(w0, g.y, z.y); z.z = fmaf(w0, g.z, z.z); z.w = fmaf(w0, g.w, z.w);
    if (lat.g1) {
      float4 h = __ldg(reinterpret_cast<const float4*>(lat.g1 + off));
      float w1 = w * lat.tw1;
      z.x = fmaf(w1, h.x, z.x); z.y = fmaf(w1, h.y, z.y); z.z = fmaf(w1, h.z, z.z); z.w = fmaf(w1, h.w, z.w);
    }
  }
  return z;
}

// Gradient w.r.t. p of channels f..f+3 of the latent vector; gx/gy/gz hold
// d z_{f+i} / d p_x etc.
__device__ __forceinline__ void latent4_grad(const Latent& lat, const Cell& c, int f, float4& gx, float4& gy,
                                             float4& gz) {
  gx = gy = gz = make_float4(0.f, 0.f, 0.f, 0.f);
  const float s = (float)(lat.R - 1);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    float wx = dx ? c.fx : 1.0f - c.fx, wy = dy ? c.fy : 1.0f - c.fy, wz = dz ? c.fz : 1.0f - c.fz;
    float ax = (dx ? s : -s) * wy * wz, ay = wx * (dy ? s : -s) * wz, az = wx * wy * (dz ? s : -s);
    int off = c.base + dx * c.sx + dy * c.sy + dz * c.sz + f;
    float4 g = __ldg(reinterpret_cast<const float4*>(lat.g0 + off));
    if (lat.g1) {
      float4 h = __ldg(reinterpret_cast<const float4*>(lat.g1 + off));
      g = make_float4(lat.tw0 * g.x + lat.tw1 * h.x, lat.tw0 * g.y + lat.tw1 * h.y, lat.tw0 * g.z + lat.tw1 * h.z,
                      lat.tw0 * g.w + lat.tw1 * h.w);
    }
    gx.x = fmaf(ax, g.x, gx.x); gx.y = fmaf(ax, g.y, gx.y); gx.z = fmaf(ax, g.z, gx.z); gx.w = fmaf(ax, g.w, gx.w);
    gy.x = fmaf(ay, g.x, gy.x); gy.y = fmaf(ay, g.y, gy.y); gy.z = fmaf(ay, g.z, gy.z); gy.w = fmaf(ay, g.w, gy.w);
    gz.x = fmaf(az, g.x, gz.x); gz.y = fmaf(az, g.y, gz.y); gz.z = fmaf(az, g.z, gz.z); gz.w = fmaf(az, g.w, gz.w);
  }
}

// sin and cos of the Fourier argument e = F_k . p (Eq. 2) with e carried to
// about twice FP32 precision: each product split exactly into hi + lo by an
// FMA, the three products summed with error-free two-sums, then
// sin(hi + lo) = sin hi + lo cos hi and cos(hi + lo) = cos hi - lo sin hi.
// A plain FP32 dot product would lose |e| * 2^-24 of the argument, which for
// the high NeRF octaves (|e| in the thousands) dominates the error; the
// rounded-to-nearest intrinsics keep the compiler from contracting the steps.
// pl is the low part of a position carried as a pair p + pl (the render's
// sample positions); F_k . pl joins the low part of the argument.
__device__ __forceinline__ void fourier_sincos(const float* f, float3 p, float& s, float& c,
                                               float3 pl = make_float3(0.f, 0.f, 0.f)) {
  const float p0 = __fmul_rn(f[0], p.x), e0 = fmaf(f[0], p.x, -p0);
  const float p1 = __fmul_rn(f[1], p.y), e1 = fmaf(f[1], p.y, -p1);
  const float p2 = __fmul_rn(f[2], p.z), e2 = fmaf(f[2], p.z, -p2);
  const float s1 = __fadd_rn(p0, p1);
  const float b1 = __fsub_rn(s1, p0);
  const float t1 = __fadd_rn(__fsub_rn(p0, __fsub_rn(s1, b1)), __fsub_rn(p1, b1));
  const float hi = __fadd_rn(s1, p2);
  const float b2 = __fsub_rn(hi, s1);
  const float t2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(hi, b2)), __fsub_rn(p2, b2));
  const float lo = e0 + e1 + e2 + t1 + t2 + (f[0] * pl.x + f[1] * pl.y + f[2] * pl.z);
  float sh, ch;
  sincosf(hi, &sh, &ch);
  s = fmaf(ch, lo, sh);
  c = fmaf(-sh, lo, ch);
}

// Full forward pass at p (+ pl, the low part of a position carried as a
// pair, which only the Fourier arguments use).  out[0..D-1]; when STASH,
// hs[i] receives the pre-activation of layer i (i = 0..l-2) for the adjoint.
template <int C, bool STASH>
__device__ __forceinline__ void forward(const float* sm, const Layout& L, int act, const Latent& lat, float3 p,
                                        float (&out)[4], float (*hs)[C], float3 pl = make_float3(0.f, 0.f, 0.f)) {
  float h[C];
  const float* W0T = sm + L.oW0T;
#pragma unroll
  for (int o = 0; o < C; ++o) h[o] = sm[L.ob0 + o];
  axpy<C>(h, W0T, p.x);
  axpy<C>(h, W0T + C, p.y);
  axpy<C>(h, W0T + 2 * C, p.z);
  const float* Fm = sm + L.oF;
  for (int k = 0; k < L.m; ++k) {
    float s, c;
    fourier_sincos(Fm + 3 * k, p, s, c, pl);
    axpy<C>(h, W0T + (3 + k) * C, s);
    axpy<C>(h, W0T + (3 + L.m + k) * C, c);
  }
  Cell cell = make_cell(lat, p);
  for (int f = 0; f < L.F; f += 4) {
    float4 z = latent4(lat, cell, f);
    const float* r = W0T + (3 + 2 * L.m + f) * C;
    axpy<C>(h, r, z.x);
    axpy<C>(h, r + C, z.y);
    axpy<C>(h, r + 2 * C, z.z);
    axpy<C>(h, r + 3 * C, z.w);
  }
  if (L.ti) axpy<C>(h, W0T + (3 + 2 * L.m + L.F) * C, lat.tin);  // Section 7 "direct" time input
  for (int i = 1; i < L.l - 1; ++i) {
    const float* base = sm + L.oHid + (i - 1) * L.hidStride;
    float a[C];
#pragma unroll
    for (int o = 0; o < C; ++o) {
      if (STASH) hs[i - 1][o] = h[o];
      a[o] = act_f(act, h[o]);
    }
#pragma unroll
    for (int o = 0; o < C; ++o) h[o] = base[C * C + o];
#pragma unroll
    for (int j = 0; j < C; ++j) axpy<C>(h, base + j * C, a[j]);
  }
  float a[C];
#pragma unroll
  for (int o = 0; o < C; ++o) {
    if (STASH) hs[L.l - 2][o] = h[o];
    a[o] = act_f(act, h[o]);
  }
#pragma unroll
  for (int d = 0; d < 4; ++d)
    out[d] = d < L.D ? sm[L.obl + d] + dotrow<C>(sm + L.oWl + d * C, a) : 0.0f;
}

// Adjoint input gradient (Section 5 "Adjoint") of sum_d s_d out_d, whose
// derivative with respect to the last hidden activation is seed[o] =
// sum_d s_d W_last[d][o] (seed = row 0 of W_last: d out_0 / d p):
// backpropagate through the hidden layers, then through layer 0's inputs:
// identity for p, cos(e) F_k / -sin(e) F_k for the Fourier features,
// trilinear Jacobian for the latent vector.
template <int C>
__device__ __forceinline__ float3 adjoint(const float* sm, const Layout& L, int act, const Latent& lat, float3 p,
                                          float (*hs)[C], const float* seed, float3 pl = make_float3(0.f, 0.f, 0.f)) {
  float delta[C];
#pragma unroll
  for (int o = 0; o < C; ++o) delta[o] = seed[o] * act_df(act, hs[L.l - 2][o]);
  for (int i = L.l - 2; i >= 1; --i) {
    const float* Wrm = sm + L.oHid + (i - 1) * L.hidStride + C * C + C;
    float g[C];
#pragma unroll
    for (int j = 0; j < C; ++j) g[j] = 0.0f;
#pragma unroll
    for (int o = 0; o < C; ++o) axpy<C>(g, Wrm + o * C, delta[o]);
#pragma unroll
    for (int j = 0; j < C; ++j) delta[j] = g[j] * act_df(act, hs[i - 1][j]);
  }
  const float* W0T = sm + L.oW0T;
  float3 dp = make_float3(dotrow<C>(W0T, delta), dotrow<C>(W0T + C, delta), dotrow<C>(W0T + 2 * C, delta));
  const float* Fm = sm + L.oF;
  for (int k = 0; k < L.m; ++k) {
    float gs = dotrow<C>(W0T + (3 + k) * C, delta);
    float gc = dotrow<C>(W0T + (3 + L.m + k) * C, delta);
    float s, c;
    fourier_sincos(Fm + 3 * k, p, s, c, pl);
    float coef = gs * c - gc * s;
    dp.x = fmaf(coef, Fm[3 * k], dp.x);
    dp.y = fmaf(coef, Fm[3 * k + 1], dp.y);
    dp.z = fmaf(coef, Fm[3 * k + 2], dp.z);
  }
  Cell cell = make_cell(lat, p);
  for (int f = 0; f < L.F; f += 4) {
    const float* r = W0T + (3 + 2 * L.m + f) * C;
    float g0 = dotrow<C>(r, delta), g1 = dotrow<C>(r + C, delta), g2 = dotrow<C>(r + 2 * C, delta),
          g3 = dotrow<C>(r + 3 * C, delta);
    float4 gx, gy, gz;
    latent4_grad(lat, cell, f, gx, gy, gz);
    dp.x += g0 * gx.x + g1 * gx.y + g2 * gx.z + g3 * gx.w;
    dp.y += g0 * gy.x + g1 * gy.y + g2 * gy.z + g3 * gy.w;
    dp.z += g0 * gz.x + g1 * gz.y + g2 * gz.z + g3 * gz.w;
  }
  return dp;
}

__device__ __forceinline__ float3 clamp_p(float3 p) { return make_float3(clamp01f(p.x), clamp01f(p.y), clamp01f(p.z)); }

// Density (and gradient for shading) at the position ph + pl (a pair) for
// shading mode SH; the finite-difference neighbours are offset as pairs.
template <int C, int SH>
__device__ __forceinline__ float sample_field(const float* sm, const Layout& L, int act, const Latent& lat, float3 p,
                                              float3 pl, float fd_h, float3& g) {
  float out[4];
  if (SH == SRN_SHADE_ADJOINT) {
    float hs[kMaxL][C];
    forward<C, true>(sm, L, act, lat, p, out, hs, pl);
    g = adjoint<C>(sm, L, act, lat, p, hs, sm + L.oWl, pl);
    return out[0];
  }
  forward<C, false>(sm, L, act, lat, p, out, nullptr, pl);
  if (SH == SRN_SHADE_HEAD) g = make_float3(out[1], out[2], out[3]);
  if (SH == SRN_SHADE_FD) {
    float gg[3];
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      float3 qh = p, ql = pl, rh = p, rl = pl;
      df::offset_axis(qh, ql, a, fd_h);
      df::offset_axis(rh, rl, a, -fd_h);
      float o1[4], o2[4];
      forward<C, false>(sm, L, act, lat, qh, o1, nullptr, ql);
      forward<C, false>(sm, L, act, lat, rh, o2, nullptr, rl);
      gg[a] = (o1[0] - o2[0]) / (2.0f * fd_h);
    }
    g = make_float3(gg[0], gg[1], gg[2]);
  }
  return out[0];
}

}  // namespace net32
}  // namespace srn
