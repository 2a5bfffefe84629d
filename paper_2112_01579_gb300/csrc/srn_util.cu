// Small utility kernels: FP32 -> FP16 parameter copies and image MSE.
#include "srn_internal.h"

namespace srn {
namespace {

__global__ void to_half_kernel(const float* __restrict__ src, __half* __restrict__ dst, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) dst[i] = __float2half_rn(src[i]);
}

// Mean squared error over the RGB channels of n RGBA pixels.  One block,
// fixed thread-to-pixel assignment and a fixed reduction tree, so the result
// is deterministic.
constexpr int kMseThreads = 1024;
__global__ void __launch_bounds__(kMseThreads) mse_kernel(const float4* __restrict__ a, const float4* __restrict__ b,
                                                          long long n, double* __restrict__ out) {
  __shared__ double part[kMseThreads];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += kMseThreads) {
    float4 x = a[i], y = b[i];
    double d0 = (double)x.x - y.x, d1 = (double)x.y - y.y, d2 = (double)x.z - y.z;
    s += d0 * d0 + d1 * d1 + d2 * d2;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = kMseThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = n > 0 ? part[0] / (3.0 * (double)n) : 0.0;
}

}  // namespace

cudaError_t launch_to_half(const float* src, __half* dst, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  to_half_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_image_mse(const float* a, const float* b, long long n, double* out, cudaStream_t s) {
  mse_kernel<<<1, kMseThreads, 0, s>>>(reinterpret_cast<const float4*>(a), reinterpret_cast<const float4*>(b), n,
                                       out);
  return cudaGetLastError();
}

}  // namespace srn
