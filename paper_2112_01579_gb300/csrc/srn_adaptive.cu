// Section 6.2 adaptive resampling: the prediction-error grid and the
// error-proportional point distribution the fit draws from.
//
// Error grid: one thread per voxel evaluates the FP32 network (the fused
// layer code of the FP32 path, weights staged in shared memory) at the
// voxel's Philox positions and averages |rho - V| in a fixed order.
//
// Distribution: every decision that turns floating point into an integer is
// an IEEE round-to-nearest operation (FP32 multiply / divide, floor), the
// rest is integer arithmetic: 16-bit voxel weights, a 64-bit exclusive
// prefix sum (block scans of 2048 weights, a scan of the block sums, an
// offset pass), and a binary search per point in the fit's point kernel.
// The result is exact and identical on every run.
#include "srn_fit.h"
#include "srn_net32.cuh"
#include "srn_sample.cuh"

namespace srn {
namespace {

using namespace net32;

constexpr int kErrThreads = 128;
constexpr int kCdfThreads = kCdfBlock / 2;  // two weights per thread

template <int C>
__global__ void __launch_bounds__(kErrThreads) error_grid_kernel(const NetDev net, const VolDev vol, int res, int spv,
                                                                 unsigned long long seed, float time,
                                                                 float* __restrict__ E, const Layout L) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  load_net<C>(sm, L, net);
  const long long nvox = (long long)res * res * res;
  const long long v = (long long)blockIdx.x * kErrThreads + threadIdx.x;
  if (v >= nvox) return;
  const Latent lat = make_latent(net, time);
  const int vx = (int)(v % res), vy = (int)((v / res) % res), vz = (int)(v / ((long long)res * res));
  const uint2 key = sample::seed_key(seed);
  float acc = 0.0f;
  for (int i = 0; i < spv; ++i) {
    const uint4 o = sample::philox4x32_10(make_uint4((unsigned)v, (unsigned)i, 0x4552u, 0u), key);
    const float3 p = make_float3(sample::voxel_coord(vx, o.x, res), sample::voxel_coord(vy, o.y, res),
                                 sample::voxel_coord(vz, o.z, res));
    float out[4];
    forward<C, false>(sm, L, net.act, lat, p, out, nullptr);
    acc += fabsf(out[0] - vol_sample(vol, p));
  }
  E[v] = acc / (float)spv;
}

template <int C>
cudaError_t error_grid_t(const NetDev& net, const VolDev& vol, int res, int spv, unsigned long long seed, float time,
                         float* E, cudaStream_t st) {
  Layout L = make_layout(net, false);
  const size_t smem = (size_t)L.total * sizeof(float);
  auto k = error_grid_kernel<C>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long nvox = (long long)res * res * res;
  k<<<(unsigned)((nvox + kErrThreads - 1) / kErrThreads), kErrThreads, smem, st>>>(net, vol, res, spv, seed, time, E,
                                                                                   L);
  return cudaGetLastError();
}

__global__ void error_max_kernel(const float* __restrict__ E, long long n, unsigned int* flags) {
  unsigned int mx = 0u, bad = 0u;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float e = E[i];
    if (!(e >= 0.0f) || isinf(e)) bad = 1u;
    else mx = max(mx, __float_as_uint(e));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(flags, 1u);
    atomicMax(flags + 1, mx);
  }
}

// 16-bit weight of one voxel: floor(E * (65535 / max)) in FP32, clamped.
__device__ __forceinline__ unsigned long long voxel_weight(float e, float scale) {
  const float f = floorf(__fmul_rn(e, scale));
  return f >= 65535.0f ? 65535ull : (unsigned long long)f;
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-local inclusive prefix of the weights into S[i + 1], block total to
// bsum[block].
__global__ void __launch_bounds__(kCdfThreads) cdf_block_kernel(const float* __restrict__ E, long long n,
                                                                const unsigned int* flags,
                                                                unsigned long long* __restrict__ S,
                                                                unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long wsum[kCdfThreads / 32];
  const float mx = __uint_as_float(flags[1]);
  const float scale = mx > 0.0f ? __fdiv_rn(65535.0f, mx) : 0.0f;
  const long long base = (long long)blockIdx.x * kCdfBlock;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long i0 = base + 2 * tid, i1 = i0 + 1;
  const unsigned long long q0 = i0 < n ? voxel_weight(E[i0], scale) : 0ull;
  const unsigned long long q1 = i1 < n ? voxel_weight(E[i1], scale) : 0ull;
  unsigned long long x = warp_incl_scan(q0 + q1, lane);
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kCdfThreads / 32 ? wsum[lane] : 0ull;
    w = warp_incl_scan(w, lane);
    if (lane < kCdfThreads / 32) wsum[lane] = w;
  }
  __syncthreads();
  const unsigned long long before = (warp > 0 ? wsum[warp - 1] : 0ull) + x - (q0 + q1);
  if (i0 < n) S[i0 + 1] = before + q0;
  if (i1 < n) S[i1 + 1] = before + q0 + q1;
  if (tid == kCdfThreads - 1) bsum[blockIdx.x] = wsum[kCdfThreads / 32 - 1];
}

// Exclusive scan of the block totals in place (one block, sequential runs
// per thread).
__global__ void __launch_bounds__(1024) cdf_bsum_kernel(unsigned long long* bsum, int nb) {
  __shared__ unsigned long long wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (nb + 1023) / 1024;
  const int b0 = tid * per;
  unsigned long long run = 0ull;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) run += bsum[b0 + k];
  unsigned long long x = warp_incl_scan(run, lane);
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) wsum[lane] = warp_incl_scan(wsum[lane], lane);
  __syncthreads();
  unsigned long long off = (warp > 0 ? wsum[warp - 1] : 0ull) + x - run;
  for (int k = 0; k < per; ++k) {
    if (b0 + k < nb) {
      const unsigned long long v = bsum[b0 + k];
      bsum[b0 + k] = off;
      off += v;
    }
  }
}

__global__ void cdf_add_kernel(unsigned long long* __restrict__ S, long long n,
                               const unsigned long long* __restrict__ bsum) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) S[0] = 0ull;
  if (i < n) S[i + 1] += bsum[i / kCdfBlock];
}

__global__ void fit_points_kernel(const unsigned long long* S, int res, unsigned long long seed, int step, int n,
                                  float* __restrict__ pts) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float3 p = sample::fit_point(S, res, seed, step, j, n);
  pts[3 * (size_t)j] = p.x;
  pts[3 * (size_t)j + 1] = p.y;
  pts[3 * (size_t)j + 2] = p.z;
}

}  // namespace

cudaError_t launch_error_grid(const NetDev& net, const VolDev& vol, int res, int spv, unsigned long long seed,
                              float time, float* E, cudaStream_t st) {
  if (net.c == 48) return error_grid_t<48>(net, vol, res, spv, seed, time, E, st);
  if (net.c == 64) return error_grid_t<64>(net, vol, res, spv, seed, time, E, st);
  return error_grid_t<32>(net, vol, res, spv, seed, time, E, st);
}

cudaError_t launch_error_max(const float* E, long long n, unsigned int* flags, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  error_max_kernel<<<(unsigned)blocks, 256, 0, st>>>(E, n, flags);
  return cudaGetLastError();
}

cudaError_t launch_build_cdf(const float* E, long long n, const unsigned int* flags, unsigned long long* S,
                             unsigned long long* bsum, cudaStream_t st) {
  const long long nb = (n + kCdfBlock - 1) / kCdfBlock;
  cdf_block_kernel<<<(unsigned)nb, kCdfThreads, 0, st>>>(E, n, flags, S, bsum);
  cdf_bsum_kernel<<<1, 1024, 0, st>>>(bsum, (int)nb);
  cdf_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, n, bsum);
  return cudaGetLastError();
}

cudaError_t launch_fit_points(const unsigned long long* S, int res, unsigned long long seed, int step, int n,
                              float* pts, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  fit_points_kernel<<<(n + 255) / 256, 256, 0, st>>>(S, res, seed, step, n, pts);
  return cudaGetLastError();
}

}  // namespace srn
