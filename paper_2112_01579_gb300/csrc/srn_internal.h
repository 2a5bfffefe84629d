// Internal declarations shared by the CUDA translation units of the library.
// Not part of the public C ABI (include/srn.h).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "srn.h"

namespace srn {

// Transfer function copied into kernel parameters (Section 3 TF mapping).
struct TFDev {
  int n;
  float opacity_scale;
  float pos[SRN_MAX_TF_POINTS];
  float4 rgba[SRN_MAX_TF_POINTS];
};

// Network description as seen by kernels.  Layer i maps d_i -> d_{i+1} with
// d_0 = 3 + 2m + F, hidden width c, output D (Section 3 layer equation).
struct NetDev {
  const float* grid;     // fp32 [nkey][R][R][R][F]
  const __half* grid_h;  // fp16 copy (FP16 path)
  const float* fourier;  // [m][3]
  const float* W;        // packed row-major layers
  const __half* W_h;     // fp16 copy of W
  const float* b;        // packed biases
  int R, F, m, l, c, D, act, nkey;
  int ti;  // 1: time is one more input after the latent vector
  int gq;  // 1: the FP16 path reads the 8-bit grid
  const uint8_t* grid_q;  // 8-bit codes
  const float* grid_qp;   // [F][2] per-channel lo, step
  // FP16 path: the FP16 latent grid holds G 2^-k (k = *grid_exp >= 0, chosen
  // by srn_sync_half from max |G| so that the FP16 latent vector stays below
  // 2^15); the layer-0 weights of the latent columns are staged times 2^k.
  const int* grid_exp;
  float key_times[SRN_MAX_KEYFRAMES];
};

// Camera frame of a pinhole camera, computed on the host in FP64 from the
// srn_camera (forward f = normalize(target - eye), right r = normalize(f x
// up), up' = r x f, th = tan(fovy / 2), tha = th W / H) and stored as FP32
// pairs value = hi + lo: the FP32 render builds its rays in double-float
// arithmetic from the pairs, the other kernels use the FP32 parts.
struct CamDev {
  float eye[3];
  float f[3], r[3], u[3];     // hi parts
  float fl[3], rl[3], ul[3];  // lo parts
  float th[2], tha[2];        // hi, lo
};

// One render batch: n_times x n_views frames of H x W pixels.
struct BatchDev {
  CamDev cams[SRN_MAX_VIEWS];
  float times[SRN_MAX_TIMES];
  int n_views, n_times;
  int W, H;
  float step, et;
  int shading;
  float fd_h;
  TFDev tf;
  float* out;                     // [n_times][n_views][H][W][4]
  unsigned long long* samples;    // nullable
  int stall_test;                 // test of the timeout path: the tensor-core render issues no MMA
};

// Dense volume source for the plain DVR.
struct VolDev {
  const float* vol;  // [nz][ny][nx]
  int nx, ny, nz;
};

// Launchers (return the cudaGetLastError of the launch).
cudaError_t launch_render_fp32(const NetDev& net, const BatchDev& b, cudaStream_t s);
cudaError_t launch_dvr_dense(const VolDev& v, const BatchDev& b, cudaStream_t s);
// mode 0: out[n][D]; 1: rho[n] + grad[n][3]; 2: grad[n][3] = sum_d dout[n][d] d out_d / d p
cudaError_t launch_eval_fp32(const NetDev& net, const float* pts, int n, float time, float* out, float* grad,
                             int mode, cudaStream_t s, const float* dout = nullptr);
bool render_fp32_supported(int width);

// FP16 tensor-core render (tcgen05 / TMEM).
cudaError_t launch_render_mma(const NetDev& net, const BatchDev& b, unsigned long long* ray_counter,
                              unsigned int* status, cudaStream_t s);
bool render_mma_supported(const NetDev& net, int shading);
bool eval_mma_supported(const NetDev& net);
cudaError_t launch_eval_mma(const NetDev& net, const float* pts, long long n, float time, float* out,
                            unsigned long long* ray_counter, unsigned int* status, cudaStream_t s);
// Density and adjoint input gradient at n points on the tensor cores (the
// render's adjoint MMAs; width 32, density output, at most four layers).
bool density_grad_mma_supported(const NetDev& net);
cudaError_t launch_density_grad_mma(const NetDev& net, const float* pts, long long n, float time, float* rho,
                                    float* grad, unsigned long long* ray_counter, unsigned int* status,
                                    cudaStream_t s);

// Conversions and small utilities.
cudaError_t launch_to_half(const float* src, __half* dst, size_t n, cudaStream_t s);
// FP16 latent grid with power-of-two scaling: exp_out[0] = k = max(0, e - 15)
// for max |grid| <= 2^e, then dst = fp16(grid 2^-k).  exp_out[1] is scratch
// (the bits of max |grid|, reduced by all blocks with one atomicMax each); the
// conversion kernel computes k from it and writes exp_out[0].
cudaError_t launch_grid_to_half_scaled(const float* grid, __half* dst, size_t n, int* exp_out, cudaStream_t s);
cudaError_t launch_quantize_grid(const float* grid, size_t n_vert, int F, uint8_t* q, float* qp, cudaStream_t s);
cudaError_t launch_image_mse(const float* a, const float* b, long long n, double* out, cudaStream_t s);
cudaError_t launch_density_mse(const float* a, const float* b, long long n, double* out, cudaStream_t s);
cudaError_t launch_image_ssim(const float* a, const float* b, int W, int H, double* out, cudaStream_t s);
cudaError_t launch_resample(const float* src, const int sdims[3], float* dst, const int ddims[3], cudaStream_t s);
bool lowpass_supported(const int dims[3], int M);
cudaError_t launch_lowpass_resample(const float* vol, const int dims[3], int M, float* tmp, float* out,
                                    cudaStream_t s);

// Layer shapes of a network.
inline int net_d0(const NetDev& n) { return 3 + 2 * n.m + n.F + n.ti; }
inline size_t net_weight_count(const NetDev& n) {
  size_t t = (size_t)n.c * net_d0(n);
  t += (size_t)(n.l - 2) * n.c * n.c;
  t += (size_t)n.D * n.c;
  return t;
}
inline size_t net_bias_count(const NetDev& n) { return (size_t)(n.l - 1) * n.c + n.D; }
inline size_t net_grid_count(const NetDev& n) { return (size_t)n.nkey * n.R * n.R * n.R * n.F; }

}  // namespace srn
