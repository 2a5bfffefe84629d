// Double-float arithmetic (a value carried as an unevaluated FP32 pair
// hi + lo, |lo| <= ulp(hi) / 2, about 44 significant bits) for the ray
// geometry of the FP32 CUDA-core render: pixel directions, box entry / exit
// and sample positions.  A sample position in plain FP32 carries a rounding
// error of a few 2^-24, which high Fourier octaves (2 pi 2^j p with j up to
// 9) and steep networks turn into image errors above the FP32 path's 1e-5
// bound; with the position carried as a pair, the Fourier arguments are
// formed from hi + lo and the only remaining position error is the rounding
// of p itself to FP32 where the network takes it as an input.
//
// The building blocks are the error-free transformations of Knuth (TwoSum,
// The Art of Computer Programming Vol. 2, 4.2.2) and Dekker (FastTwoSum and
// the double-length arithmetic of "A floating-point technique for extending
// the available precision", Numer. Math. 18, 1971), with the product error
// taken from one FMA.  The __f*_rn intrinsics keep the compiler from
// contracting or reassociating the steps.  The leading quotient and square
// root come from CUDA's correctly rounded FP32 division and sqrtf.
#pragma once

#include "srn_internal.h"

namespace srn {
namespace df {

struct F2 {
  float h, l;
};

__device__ __forceinline__ F2 make(float h) { return F2{h, 0.0f}; }

// a + b exactly as a pair (Knuth TwoSum).
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return F2{s, e};
}

// a + b exactly as a pair when |a| >= |b| or a == 0 (Dekker FastTwoSum).
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * b exactly as a pair (the FMA gives the rounding error of the product).
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return F2{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
  F2 s = two_sum(a.h, b.h);
  const F2 t = two_sum(a.l, b.l);
  s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}

__device__ __forceinline__ F2 neg(F2 a) { return F2{-a.h, -a.l}; }
__device__ __forceinline__ F2 sub(F2 a, F2 b) { return add(a, neg(b)); }

__device__ __forceinline__ F2 mul(F2 a, F2 b) {
  F2 p = two_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ F2 mul(F2 a, float b) {
  F2 p = two_prod(a.h, b);
  p.l = __fmaf_rn(a.l, b, p.l);
  return fast_two_sum(p.h, p.l);
}

// a / b: leading quotient, the exact residual a - q b, one correction.
__device__ __forceinline__ F2 div(F2 a, F2 b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const F2 r = sub(a, mul(b, q1));
  const float q2 = __fdiv_rn(r.h, b.h);
  return fast_two_sum(q1, q2);
}

// sqrt(a), a > 0: leading root, the exact residual a - s^2, one correction.
__device__ __forceinline__ F2 sqrt(F2 a) {
  const float s = __fsqrt_rn(a.h);
  const F2 r = sub(a, two_prod(s, s));
  return fast_two_sum(s, __fdiv_rn(r.h, __fmul_rn(2.0f, s)));
}

__device__ __forceinline__ bool lt(F2 a, F2 b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ F2 max(F2 a, F2 b) { return lt(a, b) ? b : a; }
__device__ __forceinline__ F2 min(F2 a, F2 b) { return lt(a, b) ? a : b; }

// Clamp to [0, 1] (the network domain).
__device__ __forceinline__ F2 clamp01(F2 a) {
  if (a.h < 0.0f || (a.h == 0.0f && a.l < 0.0f)) return F2{0.0f, 0.0f};
  if (a.h > 1.0f || (a.h == 1.0f && a.l > 0.0f)) return F2{1.0f, 0.0f};
  return a;
}

// A ray as pairs: origin o (exact FP32 eye) shifted by 0.5 into network
// coordinates, direction d, entry / exit t0, t1.
struct Ray {
  F2 o5[3];  // eye + 0.5
  F2 d[3];
  F2 t0, t1;
};

// Pinhole ray through the centre of pixel (px, py) from the camera frame
// (host-computed in FP64, stored as pairs), row 0 at the top; then the box
// [-0.5, 0.5]^3 entry and exit.  Returns false on a miss (tie = miss).
__device__ __forceinline__ bool ray_setup(const CamDev& c, int W, int H, int px, int py, Ray& r) {
  // sx = ((2 px + 1) / W - 1) tan(fovy / 2) W / H, sy = (1 - (2 py + 1) / H) tan(fovy / 2)
  const F2 qx = div(make((float)(2 * px + 1)), make((float)W));
  const F2 qy = div(make((float)(2 * py + 1)), make((float)H));
  const F2 sx = mul(add(qx, make(-1.0f)), F2{c.tha[0], c.tha[1]});
  const F2 sy = mul(add(make(1.0f), neg(qy)), F2{c.th[0], c.th[1]});
  F2 dir[3];
  F2 n2 = make(0.0f);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dir[a] = add(F2{c.f[a], c.fl[a]}, add(mul(sx, F2{c.r[a], c.rl[a]}), mul(sy, F2{c.u[a], c.ul[a]})));
    n2 = add(n2, mul(dir[a], dir[a]));
  }
  const F2 nd = sqrt(n2);
  F2 tn = make(-INFINITY), tf = make(INFINITY);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r.d[a] = div(dir[a], nd);
    r.o5[a] = two_sum(c.eye[a], 0.5f);
    if (r.d[a].h == 0.0f) {
      if (c.eye[a] < -0.5f || c.eye[a] > 0.5f) return false;
      continue;
    }
    F2 ta = div(two_sum(-0.5f, -c.eye[a]), r.d[a]);
    F2 tb = div(two_sum(0.5f, -c.eye[a]), r.d[a]);
    if (lt(tb, ta)) {
      const F2 s = ta;
      ta = tb;
      tb = s;
    }
    tn = max(tn, ta);
    tf = min(tf, tb);
  }
  r.t0 = max(tn, make(0.0f));
  r.t1 = tf;
  return lt(r.t0, r.t1);
}

// Segment k of the march, [t0 + k step, min(t0 + (k+1) step, t1)]: false when
// it starts at or beyond t1; otherwise its length and the position of its
// midpoint, clamped to [0, 1]^3, as pairs (ph + pl).
__device__ __forceinline__ bool segment(const Ray& r, int k, float step, float& len, float3& ph, float3& pl) {
  const F2 ta = add(r.t0, two_prod((float)k, step));
  if (!lt(ta, r.t1)) return false;
  const F2 tb = min(add(r.t0, two_prod((float)(k + 1), step)), r.t1);
  const F2 dt = sub(tb, ta);
  len = dt.h + dt.l;
  const F2 s = add(ta, tb);
  const F2 tm = F2{0.5f * s.h, 0.5f * s.l};  // exact halving
  float hh[3], ll[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const F2 p = clamp01(add(r.o5[a], mul(r.d[a], tm)));
    hh[a] = p.h;
    ll[a] = p.l;
  }
  ph = make_float3(hh[0], hh[1], hh[2]);
  pl = make_float3(ll[0], ll[1], ll[2]);
  return true;
}

// (ph + pl) + h along one axis, clamped to [0, 1]: the finite-difference
// neighbours of a sample.
__device__ __forceinline__ void offset_axis(float3& ph, float3& pl, int axis, float h) {
  float* hp = axis == 0 ? &ph.x : (axis == 1 ? &ph.y : &ph.z);
  float* lp = axis == 0 ? &pl.x : (axis == 1 ? &pl.y : &pl.z);
  const F2 v = clamp01(add(F2{*hp, *lp}, make(h)));
  *hp = v.h;
  *lp = v.l;
}

}  // namespace df
}  // namespace srn
