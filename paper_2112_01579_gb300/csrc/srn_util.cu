// Small utility kernels: FP32 -> FP16 parameter copies, image / density MSE,
// and the equal-memory low-pass baseline of Section 6.2 (Gaussian filter and
// vertex-aligned trilinear resampling of a dense volume).
#include "srn_device.cuh"

namespace srn {
namespace {

__global__ void to_half_kernel(const float* __restrict__ src, __half* __restrict__ dst, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) dst[i] = __float2half_rn(src[i]);
}

// Mean squared differences (image RGB, density) in FP64 over every SM, and
// still deterministic: element range b of kMseParts fixed, equal ranges
// (they depend on n only) is summed by block b in a fixed thread order and
// tree, and one block adds the kMseParts partial sums in a fixed tree.  The
// partial sums live in stream-ordered scratch of kMseParts doubles.
constexpr int kMseThreads = 256;
constexpr int kMseParts = 1024;

template <int V>  // V = 4: RGBA pixels, RGB compared; V = 1: scalars
__device__ __forceinline__ double sq_diff(const float* __restrict__ a, const float* __restrict__ b, long long i) {
  if constexpr (V == 4) {
    const float4 x = reinterpret_cast<const float4*>(a)[i], y = reinterpret_cast<const float4*>(b)[i];
    const double d0 = (double)x.x - y.x, d1 = (double)x.y - y.y, d2 = (double)x.z - y.z;
    return d0 * d0 + d1 * d1 + d2 * d2;
  } else {
    const double d = (double)a[i] - (double)b[i];
    return d * d;
  }
}

template <int NT>
__device__ __forceinline__ double block_sum(double s, double* part) {
  part[threadIdx.x] = s;
  __syncthreads();
#pragma unroll 1
  for (int w = NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  return part[0];
}

template <int V>
__global__ void __launch_bounds__(kMseThreads) mse_part_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                                               long long n, double* __restrict__ parts) {
  __shared__ double part[kMseThreads];
  const long long per = (n + kMseParts - 1) / kMseParts;
  const long long lo = (long long)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += kMseThreads) s += sq_diff<V>(a, b, i);
  const double t = block_sum<kMseThreads>(s, part);
  if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kMseParts) mse_final_kernel(const double* __restrict__ parts, double denom,
                                                              double* __restrict__ out) {
  __shared__ double part[kMseParts];
  const double t = block_sum<kMseParts>(parts[threadIdx.x], part);
  if (threadIdx.x == 0) *out = denom > 0.0 ? t / denom : 0.0;
}

template <int V>
cudaError_t launch_mse(const float* a, const float* b, long long n, double denom, double* out, cudaStream_t s) {
  double* parts = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&parts, kMseParts * sizeof(double), s);
  if (e != cudaSuccess) return e;
  mse_part_kernel<V><<<kMseParts, kMseThreads, 0, s>>>(a, b, n, parts);
  mse_final_kernel<<<1, kMseParts, 0, s>>>(parts, denom, out);
  e = cudaGetLastError();
  const cudaError_t f = cudaFreeAsync(parts, s);
  return e != cudaSuccess ? e : f;
}

// SSIM (Wang, Bovik, Sheikh, Simoncelli 2004) of two H x W RGBA images over
// the RGB channels: 11 x 11 Gaussian window (sigma 1.5, normalised), K1
// 0.01, K2 0.03, dynamic range 1, windows entirely inside the image, mean
// over channels and window centres.  FP64 throughout: FP32 inputs widen
// exactly and their products are exact in FP64, so the local variances
// sxx - mx^2 lose nothing to cancellation beyond FP64 rounding.  A block
// owns a 32 x 8 tile of window centres: it stages the tile's 42 x 18 halo of
// one channel in shared memory, filters rows, then columns, and sums its
// SSIM values in a fixed tree; the per-block sums are added in block order.
constexpr int kSsimTX = 32, kSsimTY = 8, kSsimR = 5;
constexpr int kSsimHX = kSsimTX + 2 * kSsimR, kSsimHY = kSsimTY + 2 * kSsimR;

__global__ void __launch_bounds__(kSsimTX * kSsimTY) ssim_tile_kernel(const float4* __restrict__ a,
                                                                      const float4* __restrict__ b, int W, int H,
                                                                      double* __restrict__ parts) {
  __shared__ double w[2 * kSsimR + 1];
  __shared__ double va[kSsimHY][kSsimHX], vb[kSsimHY][kSsimHX];
  __shared__ double hs[5][kSsimHY][kSsimTX];  // row-filtered a, b, aa, bb, ab
  __shared__ double part[kSsimTX * kSsimTY];
  const int tid = threadIdx.x;
  if (tid == 0) {
    double t[2 * kSsimR + 1], sum = 0.0;
    for (int k = 0; k <= 2 * kSsimR; ++k) {
      t[k] = exp(-0.5 * (double)((k - kSsimR) * (k - kSsimR)) / (1.5 * 1.5));
      sum += t[k];
    }
    for (int k = 0; k <= 2 * kSsimR; ++k) w[k] = t[k] / sum;
  }
  const int Wv = W - 2 * kSsimR, Hv = H - 2 * kSsimR;  // window centres (> 0 here)
  const int x0 = blockIdx.x * kSsimTX, y0 = blockIdx.y * kSsimTY;  // first centre, minus kSsimR
  const int ox = tid % kSsimTX, oy = tid / kSsimTX;
  const bool valid = x0 + ox < Wv && y0 + oy < Hv;
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
  double acc = 0.0;
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int i = tid; i < kSsimHX * kSsimHY; i += kSsimTX * kSsimTY) {
      const int hx = i % kSsimHX, hy = i / kSsimHX;
      const int gx = min(x0 + hx, W - 1), gy = min(y0 + hy, H - 1);  // clamped: only feeds unused centres
      const float4 pa = a[(size_t)gy * W + gx], pb = b[(size_t)gy * W + gx];
      va[hy][hx] = (double)(c == 0 ? pa.x : (c == 1 ? pa.y : pa.z));
      vb[hy][hx] = (double)(c == 0 ? pb.x : (c == 1 ? pb.y : pb.z));
    }
    __syncthreads();
    for (int i = tid; i < kSsimHY * kSsimTX; i += kSsimTX * kSsimTY) {
      const int tx = i % kSsimTX, hy = i / kSsimTX;
      double m1 = 0.0, m2 = 0.0, s11 = 0.0, s22 = 0.0, s12 = 0.0;
      for (int k = 0; k <= 2 * kSsimR; ++k) {
        const double p = va[hy][tx + k], q = vb[hy][tx + k], wk = w[k];
        m1 = fma(wk, p, m1);
        m2 = fma(wk, q, m2);
        s11 = fma(wk, p * p, s11);
        s22 = fma(wk, q * q, s22);
        s12 = fma(wk, p * q, s12);
      }
      hs[0][hy][tx] = m1;
      hs[1][hy][tx] = m2;
      hs[2][hy][tx] = s11;
      hs[3][hy][tx] = s22;
      hs[4][hy][tx] = s12;
    }
    __syncthreads();
    if (valid) {
      double m1 = 0.0, m2 = 0.0, s11 = 0.0, s22 = 0.0, s12 = 0.0;
      for (int k = 0; k <= 2 * kSsimR; ++k) {
        const double wk = w[k];
        m1 = fma(wk, hs[0][oy + k][ox], m1);
        m2 = fma(wk, hs[1][oy + k][ox], m2);
        s11 = fma(wk, hs[2][oy + k][ox], s11);
        s22 = fma(wk, hs[3][oy + k][ox], s22);
        s12 = fma(wk, hs[4][oy + k][ox], s12);
      }
      const double v1 = s11 - m1 * m1, v2 = s22 - m2 * m2, cv = s12 - m1 * m2;
      acc += ((2.0 * m1 * m2 + C1) * (2.0 * cv + C2)) / ((m1 * m1 + m2 * m2 + C1) * (v1 + v2 + C2));
    }
  }
  const double t = block_sum<kSsimTX * kSsimTY>(acc, part);
  if (tid == 0) parts[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Sum of n partial sums in index order per thread, then a fixed tree.
__global__ void __launch_bounds__(kMseParts) sum_parts_kernel(const double* __restrict__ parts, long long n,
                                                              double denom, double* __restrict__ out) {
  __shared__ double part[kMseParts];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += kMseParts) s += parts[i];
  const double t = block_sum<kMseParts>(s, part);
  if (threadIdx.x == 0) *out = t / denom;
}

__global__ void set_double_kernel(double* out, double v) { *out = v; }

// One separable Gaussian pass along `axis` with clamp-to-edge: normalised
// weights exp(-k^2 / (2 sigma^2)), |k| <= ceil(3 sigma).
constexpr int kMaxTaps = 257;
__global__ void gauss_pass_kernel(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int nz,
                                  int axis, float sigma) {
  __shared__ float w[kMaxTaps];
  const int rad = (int)ceilf(3.0f * sigma);
  for (int k = threadIdx.x; k <= 2 * rad; k += blockDim.x) {
    const float t = (float)(k - rad);
    w[k] = expf(-0.5f * t * t / (sigma * sigma));
  }
  __syncthreads();
  float wsum = 0.f;
  for (int k = 0; k <= 2 * rad; ++k) wsum += w[k];
  const long long n = (long long)nx * ny * nz;
  const int dims[3] = {nx, ny, nz};
  const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long long)nx * ny);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(axis == 0 ? i % nx : (axis == 1 ? (i / nx) % ny : i / ((long long)nx * ny)));
    float acc = 0.f;
    for (int k = -rad; k <= rad; ++k) {
      const int q = min(max(c + k, 0), dims[axis] - 1);
      acc = fmaf(w[k + rad], src[i + (long long)(q - c) * stride], acc);
    }
    dst[i] = acc / wsum;
  }
}

// Vertex-aligned trilinear resampling of a volume to another grid.
__global__ void resample_kernel(VolDev src, float* __restrict__ dst, int mx, int my, int mz) {
  const long long n = (long long)mx * my * mz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((long long)mx * my));
    const float3 p = make_float3(mx > 1 ? (float)x / (float)(mx - 1) : 0.f, my > 1 ? (float)y / (float)(my - 1) : 0.f,
                                 mz > 1 ? (float)z / (float)(mz - 1) : 0.f);
    dst[i] = vol_sample(src, p);
  }
}

// Per-channel min / max of the latent grid (one block per channel, fixed
// reduction tree) and the 8-bit codes of Section 4.2.
constexpr int kQThreads = 256;
__global__ void __launch_bounds__(kQThreads) channel_range_kernel(const float* __restrict__ g, size_t n_vert, int F,
                                                                  float* __restrict__ qp) {
  __shared__ float lo_s[kQThreads], hi_s[kQThreads];
  const int f = blockIdx.x;
  float lo = INFINITY, hi = -INFINITY;
  for (size_t v = threadIdx.x; v < n_vert; v += kQThreads) {
    const float x = g[v * F + f];
    lo = fminf(lo, x);
    hi = fmaxf(hi, x);
  }
  lo_s[threadIdx.x] = lo;
  hi_s[threadIdx.x] = hi;
  __syncthreads();
  for (int w = kQThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      lo_s[threadIdx.x] = fminf(lo_s[threadIdx.x], lo_s[threadIdx.x + w]);
      hi_s[threadIdx.x] = fmaxf(hi_s[threadIdx.x], hi_s[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float step = hi_s[0] > lo_s[0] ? (hi_s[0] - lo_s[0]) / 255.0f : 1.0f;
    qp[2 * f] = lo_s[0];
    qp[2 * f + 1] = step;
  }
}

__global__ void quantize_kernel(const float* __restrict__ g, size_t n, int F, const float* __restrict__ qp,
                                uint8_t* __restrict__ q) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(i % F);
    const float c = rintf((g[i] - qp[2 * f]) / qp[2 * f + 1]);
    q[i] = (uint8_t)fminf(fmaxf(c, 0.0f), 255.0f);
  }
}

unsigned int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned int)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_density_mse(const float* a, const float* b, long long n, double* out, cudaStream_t s) {
  return launch_mse<1>(a, b, n, (double)n, out, s);
}

cudaError_t launch_resample(const float* src, const int sdims[3], float* dst, const int ddims[3], cudaStream_t s) {
  VolDev v{src, sdims[0], sdims[1], sdims[2]};
  resample_kernel<<<grid_for((long long)ddims[0] * ddims[1] * ddims[2]), 256, 0, s>>>(v, dst, ddims[0], ddims[1],
                                                                                        ddims[2]);
  return cudaGetLastError();
}

bool lowpass_supported(const int dims[3], int M) {
  for (int a = 0; a < 3; ++a) {
    const float sigma = 0.5f * (float)(dims[a] - 1) / (float)(M - 1);
    if (2 * (int)ceilf(3.0f * sigma) + 1 > kMaxTaps) return false;
  }
  return true;
}

cudaError_t launch_lowpass_resample(const float* vol, const int dims[3], int M, float* tmp, float* out,
                                    cudaStream_t s) {
  const long long n = (long long)dims[0] * dims[1] * dims[2];
  float* a = tmp;
  float* b = tmp + n;
  const float* cur = vol;
  for (int axis = 0; axis < 3; ++axis) {
    float* dst = (axis % 2 == 0) ? a : b;
    const float sigma = 0.5f * (float)(dims[axis] - 1) / (float)(M - 1);
    gauss_pass_kernel<<<grid_for(n), 256, 0, s>>>(cur, dst, dims[0], dims[1], dims[2], axis, sigma);
    cur = dst;
  }
  const int md[3] = {M, M, M};
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_resample(cur, dims, out, md, s);
}

cudaError_t launch_to_half(const float* src, __half* dst, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  to_half_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

namespace {
// max |grid| over all blocks: each block reduces its grid-stride share, then
// one atomicMax on the bits (non-negative floats order like their bits; NaN
// entries are skipped by fmaxf, as non-finite grids are reported by the
// kernels that read them).
__global__ void grid_absmax_kernel(const float* __restrict__ g, size_t n, unsigned int* __restrict__ max_bits) {
  __shared__ float red[32];
  float m = 0.0f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(g[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(max_bits, __float_as_uint(m));
  }
}

// Exponent of the FP16 latent-grid scale: the smallest k >= 0 with
// max |grid| 2^-k <= 2^15 (max |grid| = 0 or non-finite: k = 0).
__device__ __forceinline__ int grid_scale_exp(unsigned int max_bits) {
  const float m = __uint_as_float(max_bits);
  int e = 0;
  if (m > 0.0f && m <= 3.4e38f) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1): m <= 2^e
  return e > 15 ? e - 15 : 0;
}

__global__ void to_half_scaled_kernel(const float* __restrict__ src, __half* __restrict__ dst, size_t n,
                                      int* __restrict__ exp_out, const unsigned int* __restrict__ max_bits) {
  const int k = grid_scale_exp(*max_bits);
  if (blockIdx.x == 0 && threadIdx.x == 0) *exp_out = k;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) dst[i] = __float2half_rn(ldexpf(src[i], -k));
}
}  // namespace

cudaError_t launch_grid_to_half_scaled(const float* grid, __half* dst, size_t n, int* exp_out, cudaStream_t s) {
  unsigned int* max_bits = reinterpret_cast<unsigned int*>(exp_out + 1);
  cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks == 0) blocks = 1;
  if (n > 0) {
    grid_absmax_kernel<<<(unsigned)blocks, 256, 0, s>>>(grid, n, max_bits);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // with n = 0 this still writes k = 0
  to_half_scaled_kernel<<<(unsigned)blocks, 256, 0, s>>>(grid, dst, n, exp_out, max_bits);
  return cudaGetLastError();
}

cudaError_t launch_image_mse(const float* a, const float* b, long long n, double* out, cudaStream_t s) {
  return launch_mse<4>(a, b, n, 3.0 * (double)n, out, s);
}

}  // namespace srn

namespace srn {

cudaError_t launch_quantize_grid(const float* grid, size_t n_vert, int F, uint8_t* q, float* qp, cudaStream_t s) {
  channel_range_kernel<<<F, kQThreads, 0, s>>>(grid, n_vert, F, qp);
  quantize_kernel<<<grid_for((long long)(n_vert * F)), 256, 0, s>>>(grid, n_vert * F, F, qp, q);
  return cudaGetLastError();
}

cudaError_t launch_image_ssim(const float* a, const float* b, int W, int H, double* out, cudaStream_t s) {
  const int Wv = W - 2 * kSsimR, Hv = H - 2 * kSsimR;
  if (Wv <= 0 || Hv <= 0) {  // no window fits: SSIM 1 by convention
    set_double_kernel<<<1, 1, 0, s>>>(out, 1.0);
    return cudaGetLastError();
  }
  const dim3 grid((Wv + kSsimTX - 1) / kSsimTX, (Hv + kSsimTY - 1) / kSsimTY);
  const long long nb = (long long)grid.x * grid.y;
  double* parts = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&parts, (size_t)nb * sizeof(double), s);
  if (e != cudaSuccess) return e;
  ssim_tile_kernel<<<grid, kSsimTX * kSsimTY, 0, s>>>(reinterpret_cast<const float4*>(a),
                                                       reinterpret_cast<const float4*>(b), W, H, parts);
  sum_parts_kernel<<<1, kMseParts, 0, s>>>(parts, nb, 3.0 * (double)Wv * (double)Hv, out);
  e = cudaGetLastError();
  const cudaError_t f = cudaFreeAsync(parts, s);
  return e != cudaSuccess ? e : f;
}

}  // namespace srn
