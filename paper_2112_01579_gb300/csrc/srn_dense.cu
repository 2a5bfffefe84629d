// Dense-grid direct volume rendering of a float32 volume: the plain method
// the fV-SRN network stands in for, and the reference renderer of the paper's
// quality comparisons (Section 4 / 6).  Same ray march, transfer function,
// compositing and shading as the network renderer; density = trilinear
// interpolation of the volume.
#include "srn_device.cuh"

namespace srn {
namespace {

constexpr int kThreads = 128;

template <bool FD>
__global__ void __launch_bounds__(kThreads) dvr_dense_kernel(const VolDev v, const BatchDev b) {
  __shared__ TFDev tf;
  load_tf(tf, b.tf);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int tiles_x = (b.W + 7) / 8, tiles_y = (b.H + 3) / 4;
  const long long tpf = (long long)tiles_x * tiles_y;
  const long long frame = warp / tpf;
  if (frame >= (long long)b.n_times * b.n_views) return;
  const int t = (int)(warp - frame * tpf);
  const int px = (t % tiles_x) * 8 + (lane & 7), py = (t / tiles_x) * 4 + (lane >> 3);
  const int view = (int)(frame % b.n_views);
  if (px >= b.W || py >= b.H) return;

  float3 o, d;
  camera_ray(b.cams[view], b.W, b.H, px, py, o, d);
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
  unsigned int ns = 0;
  float t0, t1;
  const float hx = 1.0f / (float)(v.nx - 1), hy = 1.0f / (float)(v.ny - 1), hz = 1.0f / (float)(v.nz - 1);
  if (box_intersect(o, d, t0, t1)) {
    for (int k = 0;; ++k) {
      float ta = fmaf((float)k, b.step, t0);
      if (ta >= t1) break;
      float tb = fminf(fmaf((float)(k + 1), b.step, t0), t1);
      float len = tb - ta, tm = 0.5f * (ta + tb);
      float3 p = make_float3(clamp01f(fmaf(tm, d.x, o.x) + 0.5f), clamp01f(fmaf(tm, d.y, o.y) + 0.5f),
                             clamp01f(fmaf(tm, d.z, o.z) + 0.5f));
      float rho = vol_sample(v, p);
      ++ns;
      float4 c = tf_eval(tf, rho);
      float alpha = 1.0f - expf(-c.w * tf.opacity_scale * len);
      if (FD) {
        float3 g;
        g.x = (vol_sample(v, make_float3(clamp01f(p.x + hx), p.y, p.z)) -
               vol_sample(v, make_float3(clamp01f(p.x - hx), p.y, p.z))) / (2.0f * hx);
        g.y = (vol_sample(v, make_float3(p.x, clamp01f(p.y + hy), p.z)) -
               vol_sample(v, make_float3(p.x, clamp01f(p.y - hy), p.z))) / (2.0f * hy);
        g.z = (vol_sample(v, make_float3(p.x, p.y, clamp01f(p.z + hz))) -
               vol_sample(v, make_float3(p.x, p.y, clamp01f(p.z - hz)))) / (2.0f * hz);
        shade(c, g, d);
      }
      float w = (1.0f - A) * alpha;
      C0 = fmaf(w, c.x, C0);
      C1 = fmaf(w, c.y, C1);
      C2 = fmaf(w, c.z, C2);
      A += w;
      if (A >= b.et) break;
    }
  }
  size_t idx = ((size_t)frame * b.H + py) * b.W + px;
  reinterpret_cast<float4*>(b.out)[idx] = make_float4(C0, C1, C2, A);
  add_samples(b.samples, ns);
}

}  // namespace

cudaError_t launch_dvr_dense(const VolDev& v, const BatchDev& b, cudaStream_t s) {
  long long tiles = (long long)((b.W + 7) / 8) * ((b.H + 3) / 4) * b.n_views * b.n_times;
  long long blocks = (tiles + (kThreads / 32) - 1) / (kThreads / 32);
  if (b.shading == SRN_SHADE_NONE)
    dvr_dense_kernel<false><<<(unsigned)blocks, kThreads, 0, s>>>(v, b);
  else
    dvr_dense_kernel<true><<<(unsigned)blocks, kThreads, 0, s>>>(v, b);
  return cudaGetLastError();
}

}  // namespace srn
