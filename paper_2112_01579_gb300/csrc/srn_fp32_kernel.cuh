// FP32 CUDA-core fV-SRN kernels: ray-marching render (all shading modes)
// and point evaluation (density, adjoint input gradient).
//
// One thread per ray / point.  The network (Section 3 layer equation, Eq. 1-2
// Fourier features, Section 4.2 latent grid) is staged once per block into
// shared memory as FP32; every sample runs the whole MLP in registers, so no
// intermediate state touches global memory (the fused-network idea of
// Section 4).  Layer 0 is accumulated feature by feature as each input
// (position, sin/cos feature, latent channel) is produced, so the input
// vector itself is never materialised.
#pragma once
#include "srn_fp32.h"
#include "srn_net32.cuh"

namespace srn {
namespace fp32 {

constexpr int kThreads = 128;
using namespace net32;

// Render: each warp covers an 8 x 4 pixel tile; one thread per ray.
template <int C, int SH>
__global__ void __launch_bounds__(kThreads) render_fp32_kernel(const NetDev net, const BatchDev b, const Layout L) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  __shared__ TFDev tf;
  load_tf(tf, b.tf);
  load_net<C>(sm, L, net);

  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int tiles_x = (b.W + 7) / 8, tiles_y = (b.H + 3) / 4;
  const long long tpf = (long long)tiles_x * tiles_y;
  const long long frame = warp / tpf;
  if (frame >= (long long)b.n_times * b.n_views) return;
  const int t = (int)(warp - frame * tpf);
  const int px = (t % tiles_x) * 8 + (lane & 7), py = (t / tiles_x) * 4 + (lane >> 3);
  const int view = (int)(frame % b.n_views), ti = (int)(frame / b.n_views);
  if (px >= b.W || py >= b.H) return;

  const Latent lat = make_latent(net, b.times[ti]);
  // ray geometry in double-float arithmetic (srn_df.cuh): direction, box
  // entry / exit and sample positions carry ~44 bits, so the network sees
  // positions rounded once
  df::Ray ray;
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
  unsigned int ns = 0;
  if (df::ray_setup(b.cams[view], b.W, b.H, px, py, ray)) {
    const float3 d = make_float3(ray.d[0].h, ray.d[1].h, ray.d[2].h);
    float len;
    float3 p, pl;
    for (int k = 0; df::segment(ray, k, b.step, len, p, pl); ++k) {
      float3 g = make_float3(0.f, 0.f, 0.f);
      float rho = sample_field<C, SH>(sm, L, net.act, lat, p, pl, b.fd_h, g);
      ++ns;
      float4 c = tf_eval(tf, rho);
      float alpha = -expm1f(-c.w * tf.opacity_scale * len);
      if (SH != SRN_SHADE_NONE) shade(c, g, d);
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

// Point evaluation: mode 0 writes out[n][D]; mode 1 writes rho[n] and the
// adjoint gradient grad[n][3] (when grad is not null); mode 2 writes the
// input vector-Jacobian product grad[n][3] = sum_d dout[n][d] d out_d / d p.
template <int C, int MODE>
__global__ void __launch_bounds__(kThreads) eval_fp32_kernel(const NetDev net, const float* __restrict__ pts, int n,
                                                             float time, float* __restrict__ out,
                                                             float* __restrict__ grad,
                                                             const float* __restrict__ dout, const Layout L) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  load_net<C>(sm, L, net);
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const Latent lat = make_latent(net, time);
  float3 p = clamp_p(make_float3(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2]));
  float o[4];
  if (MODE == 0) {
    forward<C, false>(sm, L, net.act, lat, p, o, nullptr);
    for (int d = 0; d < L.D; ++d) out[(size_t)j * L.D + d] = o[d];
  } else if (MODE == 1) {
    float hs[kMaxL][C];
    forward<C, true>(sm, L, net.act, lat, p, o, hs);
    out[j] = o[0];
    if (grad) {
      float3 g = adjoint<C>(sm, L, net.act, lat, p, hs, sm + L.oWl);
      grad[3 * j] = g.x;
      grad[3 * j + 1] = g.y;
      grad[3 * j + 2] = g.z;
    }
  } else {
    float hs[kMaxL][C];
    forward<C, true>(sm, L, net.act, lat, p, o, hs);
    float seed[C];
#pragma unroll
    for (int c = 0; c < C; ++c) seed[c] = 0.0f;
    for (int d = 0; d < L.D; ++d) {
      const float s = dout[(size_t)j * L.D + d];
#pragma unroll
      for (int c = 0; c < C; ++c) seed[c] = fmaf(s, sm[L.oWl + d * C + c], seed[c]);
    }
    const float3 g = adjoint<C>(sm, L, net.act, lat, p, hs, seed);
    grad[3 * j] = g.x;
    grad[3 * j + 1] = g.y;
    grad[3 * j + 2] = g.z;
  }
}

template <int C, int SH>
cudaError_t launch_render_t(const NetDev& net, const BatchDev& b, cudaStream_t s) {
  Layout L = make_layout(net, SH == SRN_SHADE_ADJOINT);
  size_t smem = (size_t)L.total * sizeof(float);
  auto k = render_fp32_kernel<C, SH>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long long tiles = (long long)((b.W + 7) / 8) * ((b.H + 3) / 4) * b.n_views * b.n_times;
  long long blocks = (tiles + (kThreads / 32) - 1) / (kThreads / 32);
  k<<<(unsigned)blocks, kThreads, smem, s>>>(net, b, L);
  return cudaGetLastError();
}

template <int C, int MODE>
cudaError_t launch_eval_t(const NetDev& net, const float* pts, int n, float time, float* out, float* grad,
                          const float* dout, cudaStream_t s) {
  Layout L = make_layout(net, MODE != 0);
  size_t smem = (size_t)L.total * sizeof(float);
  auto k = eval_fp32_kernel<C, MODE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(n + kThreads - 1) / kThreads, kThreads, smem, s>>>(net, pts, n, time, out, grad, dout, L);
  return cudaGetLastError();
}

// Explicit instantiation of one width's render (all shading modes) or point
// evaluation (both modes).
#define SRN_FP32_RENDER(C, SH)                                                                  \
  template cudaError_t launch_render_t<C, SH>(const NetDev&, const BatchDev&, cudaStream_t);
#define SRN_FP32_EVAL(C, MODE)                                                                  \
  template cudaError_t launch_eval_t<C, MODE>(const NetDev&, const float*, int, float, float*, float*, \
                                              const float*, cudaStream_t);

}  // namespace fp32
}  // namespace srn
