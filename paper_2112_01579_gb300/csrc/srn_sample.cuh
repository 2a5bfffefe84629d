// Training-point samplers of the fit (Section 5 uniform world-space
// sampling; Section 6.2 adaptive resampling) and the Philox4x32-10
// generator they draw from.
#pragma once
#include <stdint.h>

namespace srn {
namespace sample {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of the
// Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key
// increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned int lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned int lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint2 seed_key(unsigned long long seed) {
  return make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
}

// Uniform training point j of a step: counter (j, step, 0x5352, 0), key
// (seed low, seed high); each coordinate is (word >> 8) * 2^-24.
__device__ __forceinline__ float3 uniform_point(unsigned long long seed, int step, int j) {
  const uint4 o = philox4x32_10(make_uint4((unsigned)j, (unsigned)step, 0x5352u, 0u), seed_key(seed));
  const float s = 1.0f / 16777216.0f;
  return make_float3((float)(o.x >> 8) * s, (float)(o.y >> 8) * s, (float)(o.z >> 8) * s);
}

// Coordinate inside voxel index va of res: (va + (word >> 8) 2^-24) / res
// with both operations rounded to nearest in FP32.
__device__ __forceinline__ float voxel_coord(int va, unsigned int word, int res) {
  const float u = (float)(word >> 8) * (1.0f / 16777216.0f);
  return __fdiv_rn(__fadd_rn((float)va, u), (float)res);
}

// Training point j of n under the adaptive distribution S (exclusive prefix
// sums of the integer voxel weights over res^3 voxels, S[res^3] = Q > 0):
// the voxel v with S[v] <= floor((2j + 1) Q / (2n)) < S[v + 1], offset by
// the uniform sampler's draw for (seed, step, j).
__device__ __forceinline__ float3 adaptive_point(const unsigned long long* __restrict__ S, int res,
                                                 unsigned long long seed, int step, int j, int n) {
  const long long nvox = (long long)res * res * res;
  const unsigned long long Q = S[nvox];
  const unsigned long long t = ((2ull * (unsigned long long)j + 1ull) * Q) / (2ull * (unsigned long long)n);
  long long lo = 0, hi = nvox;  // S[lo] <= t < S[hi]
  while (hi - lo > 1) {
    const long long mid = (lo + hi) >> 1;
    if (__ldg(S + mid) <= t) lo = mid;
    else hi = mid;
  }
  const int vx = (int)(lo % res), vy = (int)((lo / res) % res), vz = (int)(lo / ((long long)res * res));
  const uint4 o = philox4x32_10(make_uint4((unsigned)j, (unsigned)step, 0x5352u, 0u), seed_key(seed));
  return make_float3(voxel_coord(vx, o.x, res), voxel_coord(vy, o.y, res), voxel_coord(vz, o.z, res));
}

// The fit's point j of n: adaptive when a distribution with Q > 0 is given,
// uniform otherwise.
__device__ __forceinline__ float3 fit_point(const unsigned long long* S, int res, unsigned long long seed, int step,
                                            int j, int n) {
  if (S != nullptr && __ldg(S + (long long)res * res * res) > 0ull) return adaptive_point(S, res, seed, step, j, n);
  return uniform_point(seed, step, j);
}

}  // namespace sample
}  // namespace srn
