// Device helpers shared by the render, eval and dense-DVR kernels.
#pragma once

#include "srn_internal.h"

namespace srn {

__device__ __forceinline__ float clamp01f(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// Pinhole ray through the centre of pixel (px, py) in FP32 from the camera
// frame (host-computed, see CamDev); row 0 at the top.
__device__ __forceinline__ void camera_ray(const CamDev& c, int W, int H, int px, int py, float3& o, float3& d) {
  const float sx = (2.0f * (px + 0.5f) / W - 1.0f) * c.tha[0];
  const float sy = (1.0f - 2.0f * (py + 0.5f) / H) * c.th[0];
  const float dx = c.f[0] + sx * c.r[0] + sy * c.u[0];
  const float dy = c.f[1] + sx * c.r[1] + sy * c.u[1];
  const float dz = c.f[2] + sx * c.r[2] + sy * c.u[2];
  const float nd = sqrtf(dx * dx + dy * dy + dz * dz);
  d = make_float3(dx / nd, dy / nd, dz / nd);
  o = make_float3(c.eye[0], c.eye[1], c.eye[2]);
}

// Entry / exit of the box [-0.5, 0.5]^3; false on a miss (tie = miss).
__device__ __forceinline__ bool box_intersect(float3 o, float3 d, float& t0, float& t1) {
  float tn = -INFINITY, tf = INFINITY;
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0f) {
      if (oo[a] < -0.5f || oo[a] > 0.5f) return false;
      continue;
    }
    float ta = (-0.5f - oo[a]) / dd[a], tb = (0.5f - oo[a]) / dd[a];
    if (ta > tb) { float s = ta; ta = tb; tb = s; }
    tn = fmaxf(tn, ta);
    tf = fminf(tf, tb);
  }
  t0 = fmaxf(tn, 0.0f);
  t1 = tf;
  return t1 > t0;
}

// Piecewise-linear TF over sorted control points (TF held in shared memory).
__device__ __forceinline__ float4 tf_eval(const TFDev& tf, float rho) {
  float x = clamp01f(rho);
  if (x <= tf.pos[0]) return tf.rgba[0];
  int n = tf.n;
  if (x >= tf.pos[n - 1]) return tf.rgba[n - 1];
  int i = 0;
  while (i < n - 2 && x >= tf.pos[i + 1]) ++i;
  float f = (x - tf.pos[i]) / (tf.pos[i + 1] - tf.pos[i]);
  float4 a = tf.rgba[i], b = tf.rgba[i + 1];
  return make_float4((1.0f - f) * a.x + f * b.x, (1.0f - f) * a.y + f * b.y, (1.0f - f) * a.z + f * b.z,
                     (1.0f - f) * a.w + f * b.w);
}

// Headlight Blinn-Phong from the density gradient (Section 5 gradient as
// isosurface normal): rgb' = rgb (0.1 + 0.6 c) + 0.3 c^32, c = |g.d| / |g|.
__device__ __forceinline__ void shade(float4& col, float3 g, float3 d) {
  float gn = sqrtf(g.x * g.x + g.y * g.y + g.z * g.z);
  if (gn < 1e-6f) return;
  float c = fabsf(g.x * d.x + g.y * d.y + g.z * d.z) / gn;
  float diff = 0.1f + 0.6f * c;
  float c2 = c * c, c4 = c2 * c2, c8 = c4 * c4, c16 = c8 * c8, c32 = c16 * c16;
  float spec = 0.3f * c32;
  col.x = col.x * diff + spec;
  col.y = col.y * diff + spec;
  col.z = col.z * diff + spec;
}

// Keyframe bracket of time t (Section 7: linear interpolation in time of the
// latent grids); times outside the keyframe range clamp.
__device__ __forceinline__ void time_weights(const NetDev& n, float t, int& k0, float& f) {
  k0 = 0;
  f = 0.0f;
  if (n.nkey <= 1) return;
  if (t <= n.key_times[0]) return;
  if (t >= n.key_times[n.nkey - 1]) { k0 = n.nkey - 2; f = 1.0f; return; }
  int k = 0;
  while (k < n.nkey - 2 && t >= n.key_times[k + 1]) ++k;
  k0 = k;
  f = (t - n.key_times[k]) / (n.key_times[k + 1] - n.key_times[k]);
}

// Vertex-aligned cell of coordinate p in [0,1] on n vertices.
__device__ __forceinline__ void cell_coord(float p, int n, int& i0, float& f) {
  float g = p * (float)(n - 1);
  int i = (int)floorf(g);
  i = min(max(i, 0), n - 2);
  i0 = i;
  f = g - (float)i;
}

// Ray and frame of a flat ray index of the batch.
__device__ __forceinline__ void batch_ray(const BatchDev& b, long long ray, int& px, int& py, int& view, int& ti) {
  px = (int)(ray % b.W);
  long long r = ray / b.W;
  py = (int)(r % b.H);
  r /= b.H;
  view = (int)(r % b.n_views);
  ti = (int)(r / b.n_views);
}

// Warp-aggregated add of per-thread sample counts to a 64-bit counter.
__device__ __forceinline__ void add_samples(unsigned long long* ctr, unsigned int ns) {
  if (ctr == nullptr) return;
  unsigned int mask = __activemask();
  unsigned int tot = __reduce_add_sync(mask, ns);
  int leader = __ffs(mask) - 1;
  if ((int)(threadIdx.x & 31) == leader && tot) atomicAdd(ctr, (unsigned long long)tot);
}

// Copy a transfer function into shared memory (block-wide).
__device__ __forceinline__ void load_tf(TFDev& dst, const TFDev& src) {
  for (int i = threadIdx.x; i < SRN_MAX_TF_POINTS; i += blockDim.x) {
    dst.pos[i] = src.pos[i];
    dst.rgba[i] = src.rgba[i];
  }
  if (threadIdx.x == 0) {
    dst.n = src.n;
    dst.opacity_scale = src.opacity_scale;
  }
}

// Trilinear interpolation of a dense float32 volume [nz][ny][nx].
__device__ __forceinline__ float vol_sample(const VolDev& v, float3 p) {
  int ix, iy, iz;
  float fx, fy, fz;
  cell_coord(p.x, v.nx, ix, fx);
  cell_coord(p.y, v.ny, iy, fy);
  cell_coord(p.z, v.nz, iz, fz);
  const size_t sy = (size_t)v.nx, sz = (size_t)v.nx * v.ny;
  const float* b = v.vol + iz * sz + iy * sy + ix;
  float c000 = __ldg(b), c100 = __ldg(b + 1), c010 = __ldg(b + sy), c110 = __ldg(b + sy + 1);
  float c001 = __ldg(b + sz), c101 = __ldg(b + sz + 1), c011 = __ldg(b + sz + sy), c111 = __ldg(b + sz + sy + 1);
  float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
  return gx * gy * gz * c000 + fx * gy * gz * c100 + gx * fy * gz * c010 + fx * fy * gz * c110 +
         gx * gy * fz * c001 + fx * gy * fz * c101 + gx * fy * fz * c011 + fx * fy * fz * c111;
}

}  // namespace srn
