// World-space fit (Section 5 training setup: uniformly drawn positions, L1
// loss against the trilinear density of the volume, Adam) and the parameter
// backward of the network, FP32 throughout.
//
// Pipeline of one step (all on the caller's stream, no host sync):
//   1. point kernel: Philox4x32-10 sample (counter = point, step; uniform or
//      the Section 6.2 error-proportional distribution), ground
//      truth, forward with stashed pre-activations, loss, backward through
//      the layers.  Weight gradients: each CTA stages delta_i and v_i of its
//      128 points in shared memory and accumulates dW_i = sum_p delta v^T for
//      the entries it owns (fixed order); one partial row per CTA.  Latent
//      adjoints dz and the cell of every point go to scratch.
//      (Two-layer width-32 density networks take the tensor-core point
//      kernel of srn_fit_mma.cu instead.)
//   2. stable LSD radix sort of (cell, point) pairs, one 9-bit pass for up to
//      512 cells, else 8-bit digits: per-block per-warp digit counts, a scan
//      per digit over the blocks, stable scatter (which adds the digits'
//      prefix and, for one pass, writes the cell offsets).
//   3. latent-grid gradient without floating-point atomics: dense cells (many
//      points per cell) sum w_corner(p) * dz per (cell, corner) in one block
//      per cell, then each vertex adds its <= 8 partials; sparse cells use one
//      warp per vertex over its cells' points in sorted order.  Fixed orders
//      and butterflies throughout, so the gradient is bit-reproducible.
//   4. fixed-order reduction of the CTA partials (weights, biases, loss), in
//      the same launch as the vertex gather.
//   5. Adam over grid, weights and biases (skipped if anything is not
//      finite), refreshing the FP16 copies.
#include <algorithm>
#include <utility>

#include "srn_fit.h"
#include "srn_net32.cuh"
#include "srn_sample.cuh"

namespace srn {
namespace {

using namespace net32;

constexpr int kFitThreads = 128;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 2048;  // keys per sort block: 8 warps x 8 rounds x 32

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

struct PointArgs {
  int n;
  int mode;  // 0: fit (sample, loss); 1: backward of given points / adjoints
  const float* pts_in;
  const float* dout_in;
  unsigned long long seed;
  int step;
  float time;
  VolDev vol;
  float gw, gs;
  const unsigned long long* cdf;  // Section 6.2 adaptive distribution (null: uniform)
  int cdf_res;
  const int* step_ptr;            // step index in device memory (graph replay), else `step`
  float* pts;   // scratch out
  float* dz;
  unsigned int* key;
  unsigned int* idx;
  float* part;
  int n_entries;
  int dstride;  // stride of the staged input rows
  int stall_test;  // timeout-path test (tensor-core point kernel only)
};

// Adds the contribution of the CTA's points to the gradient entries of one
// layer: W block (dout x din at woff) and bias block (dout at boff).  Each
// sum over the CTA's points runs as four interleaved partial sums (points
// p = 4q + r) combined at the end, a fixed order.
__device__ __forceinline__ void accumulate_layer(float* sacc, const float* sdelta, int dstr_d, const float* svin,
                                                 int dstr_v, int dout, int din, int woff, int boff) {
  const int tid = threadIdx.x;
  for (int e = tid; e < dout * din; e += kFitThreads) {
    const int o = e / din, j = e - o * din;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
    for (int p = 0; p < kFitThreads; p += 4) {
      s0 = fmaf(sdelta[p * dstr_d + o], svin[p * dstr_v + j], s0);
      s1 = fmaf(sdelta[(p + 1) * dstr_d + o], svin[(p + 1) * dstr_v + j], s1);
      s2 = fmaf(sdelta[(p + 2) * dstr_d + o], svin[(p + 2) * dstr_v + j], s2);
      s3 = fmaf(sdelta[(p + 3) * dstr_d + o], svin[(p + 3) * dstr_v + j], s3);
    }
    sacc[woff + e] += (s0 + s1) + (s2 + s3);
  }
  for (int e = tid; e < dout; e += kFitThreads) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
    for (int p = 0; p < kFitThreads; p += 4) {
      s0 += sdelta[p * dstr_d + e];
      s1 += sdelta[(p + 1) * dstr_d + e];
      s2 += sdelta[(p + 2) * dstr_d + e];
      s3 += sdelta[(p + 3) * dstr_d + e];
    }
    sacc[boff + e] += (s0 + s1) + (s2 + s3);
  }
}

template <int C>
__global__ void __launch_bounds__(kFitThreads, 4) fit_point_kernel(const NetDev net, const PointArgs a, const Layout L) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int dstr_d = C + 1, dstr_v = a.dstride;
  float* sdelta = sm + L.total;
  float* svin = sdelta + kFitThreads * dstr_d;
  float* sacc = svin + kFitThreads * dstr_v;
  float* sred = sacc + ((a.n_entries + 3) & ~3);
  load_net<C>(sm, L, net);
  const int tid = threadIdx.x;
  const int step = a.step_ptr ? *a.step_ptr : a.step;
  for (int e = tid; e < a.n_entries; e += kFitThreads) sacc[e] = 0.f;

  // packed offsets of each layer's weights / biases in [W | b]
  const int d0 = L.d0, l = L.l, D = L.D;
  const int nW = C * d0 + (l - 2) * C * C + D * C;
  const Latent lat = make_latent(net, a.time);
  const float inv_n = 1.0f / (float)a.n;
  float loss_acc = 0.f;
  const int nchunks = (a.n + kFitThreads - 1) / kFitThreads;

  for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const int j = chunk * kFitThreads + tid;
    const bool valid = j < a.n;
    float3 p = make_float3(0.5f, 0.5f, 0.5f);
    float out[4] = {0.f, 0.f, 0.f, 0.f}, dout[4] = {0.f, 0.f, 0.f, 0.f};
    float hs[kMaxL][C];
    if (valid) {
      if (a.mode == 0) p = sample::fit_point(a.cdf, a.cdf_res, a.seed, step, j, a.n);
      else p = clamp_p(make_float3(a.pts_in[3 * j], a.pts_in[3 * j + 1], a.pts_in[3 * j + 2]));
      forward<C, true>(sm, L, net.act, lat, p, out, hs);
      if (a.mode == 0) {
        const float r = out[0] - vol_sample(a.vol, p);
        loss_acc += fabsf(r);
        dout[0] = sgnf(r) * inv_n;
        if (D == 4) {
          const float hh[3] = {1.0f / (float)(a.vol.nx - 1), 1.0f / (float)(a.vol.ny - 1),
                               1.0f / (float)(a.vol.nz - 1)};
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            float3 pp = p, pm = p;
            if (ax == 0) { pp.x = clamp01f(p.x + hh[0]); pm.x = clamp01f(p.x - hh[0]); }
            if (ax == 1) { pp.y = clamp01f(p.y + hh[1]); pm.y = clamp01f(p.y - hh[1]); }
            if (ax == 2) { pp.z = clamp01f(p.z + hh[2]); pm.z = clamp01f(p.z - hh[2]); }
            const float g = (vol_sample(a.vol, pp) - vol_sample(a.vol, pm)) / (2.0f * hh[ax]);
            const float ra = out[1 + ax] - a.gs * g;
            loss_acc += a.gw * fabsf(ra);
            dout[1 + ax] = a.gw * sgnf(ra) * inv_n;
          }
        }
      } else {
        for (int dd = 0; dd < D; ++dd) dout[dd] = a.dout_in[(size_t)j * D + dd];
      }
    }
    // ---- last layer (C -> D): delta = dout, input = act(h_{l-2}); the
    // activation and its derivative come from one sin/cos evaluation
    float dact[C];
#pragma unroll
    for (int o = 0; o < C; ++o) {
      float av = 0.f, dv = 0.f;
      if (valid) act_and_df(net.act, hs[l - 2][o], av, dv);
      svin[tid * dstr_v + o] = av;
      dact[o] = dv;
    }
#pragma unroll
    for (int dd = 0; dd < 4; ++dd)
      if (dd < D) sdelta[tid * dstr_d + dd] = dout[dd];
    __syncthreads();
    accumulate_layer(sacc, sdelta, dstr_d, svin, dstr_v, D, C, nW - D * C, nW + (l - 1) * C);
    __syncthreads();
    float delta[C];
#pragma unroll
    for (int jj = 0; jj < C; ++jj) {
      float g = 0.f;
      for (int dd = 0; dd < D; ++dd) g = fmaf(sm[L.oWl + dd * C + jj], dout[dd], g);
      delta[jj] = g * dact[jj];
    }
    // ---- hidden layers i = l-2 .. 1 (C -> C)
    for (int i = l - 2; i >= 1; --i) {
#pragma unroll
      for (int o = 0; o < C; ++o) {
        float av = 0.f, dv = 0.f;
        if (valid) act_and_df(net.act, hs[i - 1][o], av, dv);
        sdelta[tid * dstr_d + o] = delta[o];
        svin[tid * dstr_v + o] = av;
        dact[o] = dv;
      }
      __syncthreads();
      accumulate_layer(sacc, sdelta, dstr_d, svin, dstr_v, C, C, C * d0 + (i - 1) * C * C, nW + i * C);
      __syncthreads();
      const float* Wrm = sm + L.oHid + (i - 1) * L.hidStride + C * C + C;
      float g[C];
#pragma unroll
      for (int jj = 0; jj < C; ++jj) g[jj] = 0.f;
#pragma unroll
      for (int o = 0; o < C; ++o) axpy<C>(g, Wrm + o * C, delta[o]);
#pragma unroll
      for (int jj = 0; jj < C; ++jj) delta[jj] = g[jj] * dact[jj];
    }
    // ---- layer 0 (d0 -> C): input [p, sin(Fp), cos(Fp), z]
#pragma unroll
    for (int o = 0; o < C; ++o) sdelta[tid * dstr_d + o] = delta[o];
    {
      float* v = svin + tid * dstr_v;
      v[0] = p.x; v[1] = p.y; v[2] = p.z;
      const float* Fm = sm + L.oF;
      for (int k = 0; k < L.m; ++k) {
        const float e = Fm[3 * k] * p.x + Fm[3 * k + 1] * p.y + Fm[3 * k + 2] * p.z;
        float s, c;
        sincosf(e, &s, &c);
        v[3 + k] = s;
        v[3 + L.m + k] = c;
      }
      const Cell cell = make_cell(lat, p);
      for (int f = 0; f < L.F; f += 4) {
        const float4 z = latent4(lat, cell, f);
        v[3 + 2 * L.m + f] = z.x;
        v[3 + 2 * L.m + f + 1] = z.y;
        v[3 + 2 * L.m + f + 2] = z.z;
        v[3 + 2 * L.m + f + 3] = z.w;
      }
      if (L.ti) v[3 + 2 * L.m + L.F] = lat.tin;
      if (!valid)
        for (int q = 0; q < d0; ++q) v[q] = 0.f;
    }
    __syncthreads();
    accumulate_layer(sacc, sdelta, dstr_d, svin, dstr_v, C, d0, 0, nW);
    __syncthreads();
    if (valid) {
      const float* W0T = sm + L.oW0T;
      float4* dzj = reinterpret_cast<float4*>(a.dz + (size_t)j * L.F);
      for (int f = 0; f < L.F; f += 4) {
        const float* r = W0T + (3 + 2 * L.m + f) * C;
        dzj[f >> 2] = make_float4(dotrow<C>(r, delta), dotrow<C>(r + C, delta), dotrow<C>(r + 2 * C, delta),
                                  dotrow<C>(r + 3 * C, delta));
      }
      a.pts[3 * j] = p.x;
      a.pts[3 * j + 1] = p.y;
      a.pts[3 * j + 2] = p.z;
      int ix, iy, iz;
      float fx, fy, fz;
      cell_coord(p.x, lat.R, ix, fx);
      cell_coord(p.y, lat.R, iy, fy);
      cell_coord(p.z, lat.R, iz, fz);
      a.key[j] = (unsigned)((iz * (lat.R - 1) + iy) * (lat.R - 1) + ix);
      a.idx[j] = (unsigned)j;
    }
  }
  // ---- per-CTA partials: gradient entries, then the loss sum (fixed tree)
  float* row = a.part + (size_t)blockIdx.x * (a.n_entries + 1);
  for (int e = tid; e < a.n_entries; e += kFitThreads) row[e] = sacc[e];
  sred[tid] = loss_acc;
  __syncthreads();
  for (int w = kFitThreads / 2; w > 0; w >>= 1) {
    if (tid < w) sred[tid] += sred[tid + w];
    __syncthreads();
  }
  if (tid == 0) row[a.n_entries] = sred[0];
}

// ---------------------------------------------------------------- radix sort
// Digit counts of one sort block (8 warps x 8 rounds x 32 keys) per warp:
// equal digits within a round are grouped with __match_any_sync.  NB bins.
template <int NB>
__device__ __forceinline__ void warp_digit_counts(const unsigned int* __restrict__ keys, int n, int shift,
                                                  unsigned int (*cnt)[NB]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int base = blockIdx.x * kSortItems + w * 256;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = base + r * 32 + lane;
    const bool valid = i < n;
    const unsigned int d = valid ? (keys[i] >> shift) & (unsigned)(NB - 1) : 0xFFFFFFFFu;
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    if (valid && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
    __syncwarp();
  }
}

// hist[d * nblocks + block] = count of digit d in the block (digit-major, so
// one exclusive scan gives every (digit, block) its output offset).
template <int NB>
__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const unsigned int* __restrict__ keys, int n,
                                                                 int shift, unsigned int* __restrict__ hist,
                                                                 int nblocks) {
  __shared__ unsigned int cnt[8][NB];
  for (int i = threadIdx.x; i < 8 * NB; i += kSortThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  warp_digit_counts<NB>(keys, n, shift, cnt);
  __syncthreads();
  for (int d = threadIdx.x; d < NB; d += kSortThreads) {
    unsigned int t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += cnt[w][d];
    hist[(size_t)d * nblocks + blockIdx.x] = t;
  }
}

// Exclusive scan of m counts in place, in segments of `seg` values, one block
// per segment: tiles of 8192 values are staged coalesced in shared memory,
// each thread scans 8 consecutive values, and a block-wide scan of the thread
// sums plus a running carry links the tiles.  Segment b starts from
// carry_in[b] (the exclusive scan of the segment sums; 0 when carry_in is
// null).  Integer sums in a fixed order, so deterministic.
constexpr int kScanThreads = 1024, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

// sums[b] = sum of segment b of a.
__global__ void __launch_bounds__(kScanThreads) seg_sum_kernel(const unsigned int* __restrict__ a, int m, int seg,
                                                               unsigned int* __restrict__ sums) {
  __shared__ unsigned int wsum[32];
  const int b0 = blockIdx.x * seg, b1 = min(m, b0 + seg);
  unsigned int t = 0;
  for (int i = b0 + threadIdx.x; i < b1; i += kScanThreads) t += a[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned int w = wsum[threadIdx.x];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
    if (threadIdx.x == 0) sums[blockIdx.x] = w;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(unsigned int* __restrict__ a, int m, int seg,
                                                            const unsigned int* __restrict__ carry_in) {
  __shared__ unsigned int tile[kScanTile + kScanTile / 32];  // padded: 8-strided reads stay conflict-free
  __shared__ unsigned int part[32];
  __shared__ unsigned int carry_s;
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * seg, s1 = min(m, s0 + seg);
  if (tid == 0) carry_s = carry_in ? carry_in[blockIdx.x] : 0u;
  for (int base = s0; base < s1; base += kScanTile) {
    for (int i = tid; i < kScanTile; i += kScanThreads) {
      const int g = base + i;
      tile[i + i / 32] = g < s1 ? a[g] : 0u;
    }
    __syncthreads();
    unsigned int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const int i = tid * kScanPer + k;
      v[k] = tile[i + i / 32];
      s += v[k];
    }
    // block-wide inclusive scan of the thread sums: warp shuffles, then the
    // 32 warp totals by warp 0
    const int lane = tid & 31, warp = tid >> 5;
    unsigned int x = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) part[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned int w = part[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      part[lane] = w;
    }
    __syncthreads();
    const unsigned int incl = (warp > 0 ? part[warp - 1] : 0u) + x;
    unsigned int run = carry_s + incl - s;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const int i = tid * kScanPer + k;
      tile[i + i / 32] = run;
      run += v[k];
    }
    __syncthreads();
    for (int i = tid; i < kScanTile; i += kScanThreads) {
      const int g = base + i;
      if (g < s1) a[g] = tile[i + i / 32];
    }
    if (tid == kScanThreads - 1) carry_s += incl;
    __syncthreads();
  }
}

// Exclusive scan of one digit's counts over the sort blocks (one block per
// digit, up to kDigitThreads * kDigitPer sort blocks), in place; the digit's
// total to totals[digit].  The scatter kernel adds the exclusive scan of the
// totals itself, so one launch replaces the segmented scan of the whole
// histogram.  Integer sums in a fixed order.
constexpr int kDigitThreads = 256, kDigitPer = 4;

__global__ void __launch_bounds__(kDigitThreads) digit_scan_kernel(unsigned int* __restrict__ hist, int nblocks,
                                                                  unsigned int* __restrict__ totals) {
  __shared__ unsigned int part[kDigitThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned int* row = hist + (size_t)blockIdx.x * nblocks;
  unsigned int v[kDigitPer], s = 0;
#pragma unroll
  for (int k = 0; k < kDigitPer; ++k) {
    const int i = tid * kDigitPer + k;
    v[k] = i < nblocks ? row[i] : 0u;
    s += v[k];
  }
  unsigned int x = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) part[warp] = x;
  __syncthreads();
  unsigned int before = 0;
  for (int w = 0; w < warp; ++w) before += part[w];
  unsigned int run = before + x - s;
#pragma unroll
  for (int k = 0; k < kDigitPer; ++k) {
    const int i = tid * kDigitPer + k;
    if (i < nblocks) row[i] = run;
    run += v[k];
  }
  if (tid == kDigitThreads - 1) totals[blockIdx.x] = before + x;
}

template <int NB>
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const unsigned int* __restrict__ kin,
                                                                    const unsigned int* __restrict__ vin,
                                                                    unsigned int* __restrict__ kout,
                                                                    unsigned int* __restrict__ vout, int n, int shift,
                                                                    const unsigned int* __restrict__ scanned,
                                                                    int nblocks, unsigned int* __restrict__ cell_start,
                                                                    int n_cells,
                                                                    const unsigned int* __restrict__ totals) {
  __shared__ unsigned int cnt[8][NB];
  __shared__ unsigned int dbase[NB];  // keys of all smaller digits (0 when `scanned` is already global)
  __shared__ unsigned int wpart[kSortThreads / 32];
  if (totals) {
    // exclusive scan of the digit totals, NB / kSortThreads consecutive digits per thread
    constexpr int PER = NB / kSortThreads;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int v[PER], t = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      v[k] = totals[threadIdx.x * PER + k];
      t += v[k];
    }
    unsigned int x = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wpart[warp] = x;
    __syncthreads();
    unsigned int run = x - t;
    for (int w = 0; w < warp; ++w) run += wpart[w];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      dbase[threadIdx.x * PER + k] = run;
      run += v[k];
    }
  } else {
    for (int d = threadIdx.x; d < NB; d += kSortThreads) dbase[d] = 0u;
  }
  for (int i = threadIdx.x; i < 8 * NB; i += kSortThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  // one-pass sort (the digit is the whole cell index): the start of cell c in
  // the sorted order is the exclusive prefix of digit c, block 0's entry
  if (cell_start && blockIdx.x == 0)
    for (int c = threadIdx.x; c <= n_cells; c += kSortThreads)
      cell_start[c] = c < NB ? dbase[c] + scanned[(size_t)c * nblocks] : (unsigned int)n;
  warp_digit_counts<NB>(kin, n, shift, cnt);
  __syncthreads();
  for (int d = threadIdx.x; d < NB; d += kSortThreads) {
    unsigned int base = dbase[d] + scanned[(size_t)d * nblocks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const unsigned int c = cnt[w][d];
      cnt[w][d] = base;
      base += c;
    }
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int base = blockIdx.x * kSortItems + w * 256;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = base + r * 32 + lane;
    const bool valid = i < n;
    const unsigned int k = valid ? kin[i] : 0u;
    const unsigned int d = valid ? (k >> shift) & (unsigned)(NB - 1) : 0xFFFFFFFFu;
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid) {
      const unsigned int pos = cnt[w][d] + rank;
      kout[pos] = k;
      vout[pos] = vin[i];
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
    __syncwarp();
  }
}

// cell_start[c] = first sorted position with key >= c, for c in [0, n_cells].
__global__ void cell_start_kernel(const unsigned int* __restrict__ skeys, int n, unsigned int* __restrict__ start,
                                  int n_cells) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  const int cur = s < n ? (int)skeys[s] : n_cells;
  const int prev = s > 0 ? (int)skeys[s - 1] : -1;
  for (int c = prev + 1; c <= cur; ++c) start[c] = (unsigned int)s;
}

// One warp per grid vertex: gather w_corner(p_j) * dz_j over the points of the
// vertex's adjacent cells (fixed cell order, sorted point order, lane-strided)
// and reduce across lanes with a fixed butterfly.
struct GradArgs {
  const float* pts;
  const float* dz;
  const unsigned int* sidx;
  const unsigned int* start;
  const float* cell_part;
  int R;
  float w0, w1;
  float* g0;
  float* g1;
};

template <int F>
__device__ __forceinline__ void grid_grad_block(const GradArgs& a, int block, unsigned int* __restrict__ flag) {
  const float* __restrict__ pts = a.pts;
  const float* __restrict__ dz = a.dz;
  const unsigned int* __restrict__ sidx = a.sidx;
  const unsigned int* __restrict__ start = a.start;
  const int R = a.R;
  const float w0 = a.w0, w1 = a.w1;
  float* __restrict__ g0 = a.g0;
  float* __restrict__ g1 = a.g1;
  const long long v = ((long long)block * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= (long long)R * R * R) return;
  const int vx = (int)(v % R), vy = (int)((v / R) % R), vz = (int)(v / ((long long)R * R));
  float acc[F];
#pragma unroll
  for (int f = 0; f < F; ++f) acc[f] = 0.f;
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dzz = c >> 2;
    const int cx = vx - dx, cy = vy - dy, cz = vz - dzz;
    if (cx < 0 || cy < 0 || cz < 0 || cx > R - 2 || cy > R - 2 || cz > R - 2) continue;
    const int cell = (cz * (R - 1) + cy) * (R - 1) + cx;
    const int s0 = (int)start[cell], s1 = (int)start[cell + 1];
    for (int s = s0 + lane; s < s1; s += 32) {
      const int j = (int)sidx[s];
      int ix, iy, iz;
      float fx, fy, fz;
      cell_coord(pts[3 * j], R, ix, fx);
      cell_coord(pts[3 * j + 1], R, iy, fy);
      cell_coord(pts[3 * j + 2], R, iz, fz);
      const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dzz ? fz : 1.0f - fz);
      const float4* zz = reinterpret_cast<const float4*>(dz + (size_t)j * F);
#pragma unroll
      for (int f = 0; f < F; f += 4) {
        const float4 q = zz[f / 4];
        acc[f] = fmaf(w, q.x, acc[f]);
        acc[f + 1] = fmaf(w, q.y, acc[f + 1]);
        acc[f + 2] = fmaf(w, q.z, acc[f + 2]);
        acc[f + 3] = fmaf(w, q.w, acc[f + 3]);
      }
    }
  }
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], off);
  if (lane == 0) {
    bool bad = false;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      g0[(size_t)v * F + f] = w0 * acc[f];
      if (g1) g1[(size_t)v * F + f] = w1 * acc[f];
      bad |= !isfinite(acc[f]);
    }
    if (bad) atomicOr(flag, 1u);
  }
}

// Dense cells (many points per cell): one block of 8 warps per cell, warp c
// sums w_corner_c(p) * dz over the cell's points (sorted order, lane-strided,
// fixed butterfly) into part[cell][c][F]; vertex_gather_block then adds the
// <= 8 partials of each vertex in a fixed order.  The block stages the cell's
// points (position, dz) in shared memory 256 at a time, so each point is
// gathered from global memory once instead of once per corner; lane l still
// takes points l, l + 32, ... in order, so the sums are those of a warp
// reading global memory directly.
template <int F>
__global__ void __launch_bounds__(256) cell_corner_kernel(const float* __restrict__ pts,
                                                          const float* __restrict__ dz,
                                                          const unsigned int* __restrict__ sidx,
                                                          const unsigned int* __restrict__ start, int R,
                                                          long long n_cells, float* __restrict__ part) {
  constexpr int kChunk = 256;
  __shared__ float sp[kChunk][3];
  __shared__ float4 sz[kChunk][F / 4];
  const long long cell = blockIdx.x;
  if (cell >= n_cells) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp;
  const int dx = c & 1, dy = (c >> 1) & 1, dzz = c >> 2;
  float acc[F];
#pragma unroll
  for (int f = 0; f < F; ++f) acc[f] = 0.f;
  const int s0 = (int)start[cell], s1 = (int)start[cell + 1];
  for (int base = s0; base < s1; base += kChunk) {
    const int cnt = min(kChunk, s1 - base);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += 256) {
      const int j = (int)sidx[base + i];
      sp[i][0] = pts[3 * (size_t)j];
      sp[i][1] = pts[3 * (size_t)j + 1];
      sp[i][2] = pts[3 * (size_t)j + 2];
      const float4* zz = reinterpret_cast<const float4*>(dz + (size_t)j * F);
#pragma unroll
      for (int f = 0; f < F / 4; ++f) sz[i][f] = zz[f];
    }
    __syncthreads();
    for (int i = lane; i < cnt; i += 32) {
      int ix, iy, iz;
      float fx, fy, fz;
      cell_coord(sp[i][0], R, ix, fx);
      cell_coord(sp[i][1], R, iy, fy);
      cell_coord(sp[i][2], R, iz, fz);
      const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dzz ? fz : 1.0f - fz);
#pragma unroll
      for (int f = 0; f < F; f += 4) {
        const float4 q = sz[i][f / 4];
        acc[f] = fmaf(w, q.x, acc[f]);
        acc[f + 1] = fmaf(w, q.y, acc[f + 1]);
        acc[f + 2] = fmaf(w, q.z, acc[f + 2]);
        acc[f + 3] = fmaf(w, q.w, acc[f + 3]);
      }
    }
  }
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], off);
  if (lane == 0) {
#pragma unroll
    for (int f = 0; f < F; ++f) part[((size_t)cell * 8 + c) * F + f] = acc[f];
  }
}

template <int F>
__device__ __forceinline__ void vertex_gather_block(const GradArgs& a, int block, unsigned int* __restrict__ flag) {
  const float* __restrict__ part = a.cell_part;
  const int R = a.R;
  const float w0 = a.w0, w1 = a.w1;
  float* __restrict__ g0 = a.g0;
  float* __restrict__ g1 = a.g1;
  const long long i = (long long)block * blockDim.x + threadIdx.x;
  if (i >= (long long)R * R * R * F) return;
  const long long v = i / F;
  const int f = (int)(i - v * F);
  const int vx = (int)(v % R), vy = (int)((v / R) % R), vz = (int)(v / ((long long)R * R));
  float acc = 0.f;
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dzz = c >> 2;
    const int cx = vx - dx, cy = vy - dy, cz = vz - dzz;
    if (cx < 0 || cy < 0 || cz < 0 || cx > R - 2 || cy > R - 2 || cz > R - 2) continue;
    const long long cell = ((long long)cz * (R - 1) + cy) * (R - 1) + cx;
    acc += part[(cell * 8 + c) * F + f];
  }
  g0[i] = w0 * acc;
  if (g1) g1[i] = w1 * acc;
  if (!isfinite(acc)) atomicOr(flag, 1u);
}

// Fixed-order sum of the CTA partials: weights, biases and the loss.  A
// block covers 32 entries; its 8 warps each sum a contiguous eighth of the
// partial rows in row order, then the 8 sums are added in warp order.
struct ReduceArgs {
  const float* part;
  int n_cta, nW, nb;
  float* outW;
  float* outb;
  float* loss;
  float inv_n;
};

__device__ __forceinline__ void reduce_parts_block(const ReduceArgs& a, int block, unsigned int* __restrict__ flag) {
  __shared__ float acc[8][32];
  const float* __restrict__ part = a.part;
  const int n_cta = a.n_cta, nW = a.nW, nb = a.nb;
  float* __restrict__ outW = a.outW;
  float* __restrict__ outb = a.outb;
  float* __restrict__ loss = a.loss;
  const float inv_n = a.inv_n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = block * 32 + lane;
  const int ne = nW + nb;
  const int r0 = (int)((long long)n_cta * w / 8), r1 = (int)((long long)n_cta * (w + 1) / 8);
  float s = 0.f;
  if (e <= ne)
    for (int c = r0; c < r1; ++c) s += part[(size_t)c * (ne + 1) + e];
  acc[w][lane] = s;
  __syncthreads();
  if (w == 0 && e <= ne) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += acc[k][lane];
    if (e < nW) outW[e] = t;
    else if (e < ne) outb[e - nW] = t;
    else if (loss) {
      t *= inv_n;
      *loss = t;
    }
    if (!isfinite(t) && (e < ne || loss)) atomicOr(flag, 1u);
  }
}

// The latent-grid gradient gather and the fixed-order reduction of the
// weight partials are independent: one launch runs both, blocks
// [0, gather_blocks) gathering, the rest reducing.
template <int F, bool DENSE>
__global__ void __launch_bounds__(256) grad_tail_kernel(const GradArgs g, int gather_blocks, const ReduceArgs r,
                                                        unsigned int* __restrict__ flag) {
  if ((int)blockIdx.x < gather_blocks) {
    if (DENSE) vertex_gather_block<F>(g, blockIdx.x, flag);
    else grid_grad_block<F>(g, blockIdx.x, flag);
  } else {
    reduce_parts_block(r, blockIdx.x - gather_blocks, flag);
  }
}

__device__ __forceinline__ void adam_update(float* __restrict__ grid, float* __restrict__ W, float* __restrict__ b,
                                            const float* __restrict__ g, float* __restrict__ m,
                                            float* __restrict__ v, size_t ng, size_t nW, size_t nb, float lr_grid,
                                            float lr_net, int step, __half* __restrict__ grid_h,
                                            __half* __restrict__ W_h, const int* __restrict__ grid_exp) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int gk = (grid_h && grid_exp) ? *grid_exp : 0;
  const float t1 = (float)step + 1.0f;  // exact below 2^24; no int overflow at INT_MAX
  const float bc1 = 1.0f - powf(b1, t1), bc2 = 1.0f - powf(b2, t1);
  const size_t n = ng + nW + nb;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / bc1) / (sqrtf(vi / bc2) + eps);
    if (i < ng) {
      const float t = grid[i] - lr_grid * upd;
      grid[i] = t;
      if (grid_h) grid_h[i] = __float2half_rn(ldexpf(t, -gk));
    } else if (i < ng + nW) {
      const float t = W[i - ng] - lr_net * upd;
      W[i - ng] = t;
      if (W_h) W_h[i - ng] = __float2half_rn(t);
    } else {
      b[i - ng - nW] -= lr_net * upd;
    }
  }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias correction at step + 1) over
// [grid | weights | biases]; refreshes the FP16 copies.  Skipped entirely
// when the step produced a non-finite loss or gradient (flag bit 0,
// SRN_ERR_NONFINITE) or a bounded wait of the point kernel gave up (bit 1,
// SRN_ERR_TIMEOUT).  With the step index
// in device memory (step_ptr), the last block to finish advances it by one
// for the next step (flag[1] counts finished blocks and is reset by that block).
__global__ void adam_kernel(float* __restrict__ grid, float* __restrict__ W, float* __restrict__ b,
                            const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, size_t ng,
                            size_t nW, size_t nb, float lr_grid, float lr_net, int step_arg, int* __restrict__ step_ptr,
                            unsigned int* __restrict__ flag, unsigned int* __restrict__ status,
                            __half* __restrict__ grid_h, __half* __restrict__ W_h,
                            const int* __restrict__ grid_exp) {
  const int step = step_ptr ? *step_ptr : step_arg;
  const unsigned int f = *flag;
  if (f) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
      atomicExch(status, (unsigned int)((f & 2u) ? SRN_ERR_TIMEOUT : SRN_ERR_NONFINITE));
  } else {
    adam_update(grid, W, b, g, m, v, ng, nW, nb, lr_grid, lr_net, step, grid_h, W_h, grid_exp);
  }
  if (step_ptr) {
    __syncthreads();  // every thread of the block has read *step_ptr
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned int done = atomicAdd(flag + 1, 1u);
      if (done == gridDim.x - 1) {
        __threadfence();
        flag[1] = 0u;
        flag[0] = 0u;  // the next replayed step starts with a clear non-finite flag
        *step_ptr = (int)((unsigned int)step + 1u);
      }
    }
  }
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Steps 1-4 shared by the fit and the backward.  Writes the grid gradient
// (all keyframes) to dgrid, weights / biases to dW / db, the loss (fit) to
// loss.
cudaError_t run_backward(FitScratch& s, const NetDev& net, PointArgs pa, float* dgrid, float* dW, float* db,
                         float* loss, cudaStream_t st, unsigned int* mma_status = nullptr) {
  const int n = pa.n;
  const int nW = (int)(net_weight_count(net)), nb = (int)net_bias_count(net);
  Layout L = make_layout(net, true);
  // odd row stride: per-thread rows written at the same column hit distinct banks
  const int dstride = ((net_d0(net) > net.c ? net_d0(net) : net.c) + 1) | 1;
  pa.dstride = dstride;
  pa.n_entries = nW + nb;
  pa.pts = s.pts;
  pa.dz = s.dz;
  pa.key = s.key;
  pa.idx = s.idx;
  pa.part = s.part;
  int n_cta = std::min(s.max_cta, (n + kFitThreads - 1) / kFitThreads);
  size_t smem = sizeof(float) * ((size_t)L.total + kFitThreads * (net.c + 1) + (size_t)kFitThreads * dstride +
                                 ((pa.n_entries + 3) & ~3) + kFitThreads);
  // graph-replayed fit steps (step index in device memory) find the flag
  // cleared by the previous step's Adam kernel or by the replay set-up
  cudaError_t e = pa.step_ptr ? cudaSuccess : cudaMemsetAsync(s.flag, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  if (pa.mode == 0 && n > 0 && mma_status && fit_mma_supported(net) && s.max_cta >= fit_mma_rows_per_cta()) {
    // tensor-core point kernel: one partial row per warpgroup
    const int rows = fit_mma_rows_per_cta();
    const int grid = std::max(1, std::min({sm_count(), s.max_cta / rows, (n + 128 * rows - 1) / (128 * rows)}));
    PointArgsMma ma{n,           pa.seed, pa.step, pa.time, pa.vol, pa.cdf, pa.cdf_res, pa.step_ptr,
                    s.pts,       s.dz,    s.key,   s.idx,  s.part, s.flag, pa.stall_test};
    e = launch_fit_mma(net, ma, grid, mma_status, st);
    if (e != cudaSuccess) return e;
    n_cta = grid * rows;
  } else if (n_cta > 0) {
    auto k = fit_point_kernel<32>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<n_cta, kFitThreads, smem, st>>>(net, pa, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // sort (cell, point) by cell
  unsigned int *k_in = s.key, *v_in = s.idx, *k_out = s.key_alt, *v_out = s.idx_alt;
  int bits = 1;
  while (((size_t)1 << bits) < s.n_cells) ++bits;
  const int nblocks = (n + kSortItems - 1) / kSortItems;
  // 9-bit digits when the cell index fits one (one pass for grids up to 8^3
  // cells), else 8-bit digits
  const int dbits = s.radix_bins == 512 && bits <= 9 ? 9 : 8;
  const int hist_m = (1 << dbits) * nblocks;
  const int nseg = (hist_m + kScanTile - 1) / kScanTile;  // one 8192-value tile per scan block
  unsigned int* seg_sums = s.hist + (size_t)s.radix_bins * (size_t)((s.max_points + kSortItems - 1) / kSortItems);
  bool starts_done = false;
  for (int shift = 0; shift < bits && n > 0; shift += dbits) {
    // a single pass leaves the cell starts to the scatter kernel
    unsigned int* cs = (shift == 0 && dbits >= bits) ? s.cell_start : nullptr;
    starts_done = cs != nullptr;
    if (dbits == 9) sort_hist_kernel<512><<<nblocks, kSortThreads, 0, st>>>(k_in, n, shift, s.hist, nblocks);
    else sort_hist_kernel<256><<<nblocks, kSortThreads, 0, st>>>(k_in, n, shift, s.hist, nblocks);
    const unsigned int* totals = nullptr;
    if (nblocks <= kDigitThreads * kDigitPer) {
      // one block per digit; the scatter kernel adds the digits' prefix
      digit_scan_kernel<<<1 << dbits, kDigitThreads, 0, st>>>(s.hist, nblocks, s.digit_totals);
      totals = s.digit_totals;
    } else if (nseg > 1) {
      seg_sum_kernel<<<nseg, kScanThreads, 0, st>>>(s.hist, hist_m, kScanTile, seg_sums);
      scan_kernel<<<1, kScanThreads, 0, st>>>(seg_sums, nseg, nseg, nullptr);
      scan_kernel<<<nseg, kScanThreads, 0, st>>>(s.hist, hist_m, kScanTile, seg_sums);
    } else {
      scan_kernel<<<1, kScanThreads, 0, st>>>(s.hist, hist_m, hist_m, nullptr);
    }
    if (dbits == 9)
      sort_scatter_kernel<512><<<nblocks, kSortThreads, 0, st>>>(k_in, v_in, k_out, v_out, n, shift, s.hist, nblocks,
                                                                 cs, (int)s.n_cells, totals);
    else
      sort_scatter_kernel<256><<<nblocks, kSortThreads, 0, st>>>(k_in, v_in, k_out, v_out, n, shift, s.hist,
                                                                 nblocks, cs, (int)s.n_cells, totals);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(k_in, k_out);
    std::swap(v_in, v_out);
  }
  if (!starts_done) cell_start_kernel<<<(n + 1 + 255) / 256, 256, 0, st>>>(k_in, n, s.cell_start, (int)s.n_cells);
  // grid gradient: the gathers below write every vertex of the two bracketing
  // keyframes; other keyframes (and everything when there are no points) are zeroed
  const size_t gsz = (size_t)net.R * net.R * net.R * net.F;
  if (net.nkey > 2 || n == 0) {
    e = cudaMemsetAsync(dgrid, 0, sizeof(float) * gsz * net.nkey, st);
    if (e != cudaSuccess) return e;
  }
  int k0 = 0;
  float f = 0.f;
  {
    // keyframe bracket of the step's time (same rule as the kernels' time_weights)
    if (net.nkey > 1) {
      const float t = pa.time;
      if (t <= net.key_times[0]) { k0 = 0; f = 0.f; }
      else if (t >= net.key_times[net.nkey - 1]) { k0 = net.nkey - 2; f = 1.f; }
      else {
        while (k0 < net.nkey - 2 && t >= net.key_times[k0 + 1]) ++k0;
        f = (t - net.key_times[k0]) / (net.key_times[k0 + 1] - net.key_times[k0]);
      }
    }
  }
  const float w0 = net.nkey > 1 ? 1.0f - f : 1.0f, w1 = f;
  float* g0 = dgrid + (size_t)k0 * gsz;
  float* g1 = net.nkey > 1 ? g0 + gsz : nullptr;
  const long long n_vert = (long long)net.R * net.R * net.R;
  const int ne = nW + nb;
  const ReduceArgs ra{s.part, n_cta, nW, nb, dW, db, loss, 1.0f / (float)n};
  const int rblocks = (ne + 1 + 31) / 32;
  if (n > 0) {
    const GradArgs ga{s.pts, s.dz, v_in, s.cell_start, s.cell_part, net.R, w0, w1, g0, g1};
    const bool dense_cells = s.cell_part && (size_t)n >= 32 * s.n_cells;
    if (dense_cells) {
      const long long nw = (long long)s.n_cells * 8;
      const unsigned int cb = (unsigned int)((nw * 32 + 255) / 256);
      const int vb = (int)((n_vert * net.F + 255) / 256);
      switch (net.F) {
        case 4:
          cell_corner_kernel<4><<<cb, 256, 0, st>>>(s.pts, s.dz, v_in, s.cell_start, net.R, (long long)s.n_cells,
                                                    s.cell_part);
          grad_tail_kernel<4, true><<<vb + rblocks, 256, 0, st>>>(ga, vb, ra, s.flag);
          break;
        case 8:
          cell_corner_kernel<8><<<cb, 256, 0, st>>>(s.pts, s.dz, v_in, s.cell_start, net.R, (long long)s.n_cells,
                                                    s.cell_part);
          grad_tail_kernel<8, true><<<vb + rblocks, 256, 0, st>>>(ga, vb, ra, s.flag);
          break;
        case 16:
          cell_corner_kernel<16><<<cb, 256, 0, st>>>(s.pts, s.dz, v_in, s.cell_start, net.R, (long long)s.n_cells,
                                                     s.cell_part);
          grad_tail_kernel<16, true><<<vb + rblocks, 256, 0, st>>>(ga, vb, ra, s.flag);
          break;
        default:
          cell_corner_kernel<32><<<cb, 256, 0, st>>>(s.pts, s.dz, v_in, s.cell_start, net.R, (long long)s.n_cells,
                                                     s.cell_part);
          grad_tail_kernel<32, true><<<vb + rblocks, 256, 0, st>>>(ga, vb, ra, s.flag);
      }
    } else {
      const int gblocks = (int)((n_vert * 32 + 255) / 256);
      if (net.F == 8) grad_tail_kernel<8, false><<<gblocks + rblocks, 256, 0, st>>>(ga, gblocks, ra, s.flag);
      else if (net.F == 16) grad_tail_kernel<16, false><<<gblocks + rblocks, 256, 0, st>>>(ga, gblocks, ra, s.flag);
      else if (net.F == 4) grad_tail_kernel<4, false><<<gblocks + rblocks, 256, 0, st>>>(ga, gblocks, ra, s.flag);
      else grad_tail_kernel<32, false><<<gblocks + rblocks, 256, 0, st>>>(ga, gblocks, ra, s.flag);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    e = cudaMemsetAsync(dW, 0, sizeof(float) * nW, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(db, 0, sizeof(float) * nb, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t fit_scratch_alloc(FitScratch& s, const NetDev& net, int max_points) {
  memset(&s, 0, sizeof(s));
  s.max_points = max_points;
  if (max_points <= 0) return cudaSuccess;
  s.n_cells = (size_t)(net.R - 1) * (net.R - 1) * (net.R - 1);
  s.n_entries = net_weight_count(net) + net_bias_count(net);
  s.n_grid = net_grid_count(net);
  s.max_cta = std::min(4 * sm_count(), (max_points + kFitThreads - 1) / kFitThreads);
  const size_t n = (size_t)max_points;
  const size_t nsb = (n + kSortItems - 1) / kSortItems;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  };
  alloc((void**)&s.pts, sizeof(float) * 3 * n);
  alloc((void**)&s.dz, sizeof(float) * net.F * n);
  alloc((void**)&s.key, sizeof(unsigned int) * n);
  alloc((void**)&s.key_alt, sizeof(unsigned int) * n);
  alloc((void**)&s.idx, sizeof(unsigned int) * n);
  alloc((void**)&s.idx_alt, sizeof(unsigned int) * n);
  s.radix_bins = sort_bins(s.n_cells);
  // radix histograms, then the per-segment sums of their scan
  alloc((void**)&s.hist, sizeof(unsigned int) * (s.radix_bins * nsb + (s.radix_bins * nsb) / 8192 + 1));
  alloc((void**)&s.digit_totals, sizeof(unsigned int) * s.radix_bins);
  alloc((void**)&s.cell_start, sizeof(unsigned int) * (s.n_cells + 1));
  alloc((void**)&s.part, sizeof(float) * (size_t)s.max_cta * (s.n_entries + 1));
  alloc((void**)&s.grads, sizeof(float) * (s.n_grid + s.n_entries));
  alloc((void**)&s.flag, sizeof(unsigned int) * 4);
  if (e == cudaSuccess) e = cudaMemset(s.flag, 0, sizeof(unsigned int) * 4);  // flag[1]: Adam's block counter
  // cell keys and point indices start valid (cell 0, point 0) and are only ever
  // overwritten with valid ones, so a step whose point kernel gave up (bounded
  // wait, SRN_ERR_TIMEOUT) still sorts and gathers inside the buffers
  for (unsigned int* q : {s.key, s.key_alt, s.idx, s.idx_alt})
    if (e == cudaSuccess) e = cudaMemset(q, 0, sizeof(unsigned int) * n);
  if ((size_t)max_points >= 32 * s.n_cells) alloc((void**)&s.cell_part, sizeof(float) * s.n_cells * 8 * net.F);
  return e;
}

void fit_scratch_free(FitScratch& s) {
  void* ps[] = {s.pts, s.dz, s.key, s.key_alt, s.idx, s.idx_alt, s.hist, s.digit_totals, s.cell_start, s.part,
                s.grads, s.flag,
                s.cell_part};
  for (void* p : ps)
    if (p) cudaFree(p);
  memset(&s, 0, sizeof(s));
}

int sort_bins(size_t n_cells) { return n_cells <= 512 ? 512 : 256; }

bool fit_supported(const NetDev& net) {
  return net.c == 32 && (net.F == 4 || net.F == 8 || net.F == 16 || net.F == 32) && net.l <= kMaxL;
}

cudaError_t launch_backward(FitScratch& s, const NetDev& net, const float* pts, int n, float time, const float* dout,
                            float* dgrid, float* dW, float* db, cudaStream_t st) {
  if (!fit_supported(net)) return cudaErrorNotSupported;
  PointArgs pa{};
  pa.n = n;
  pa.mode = 1;
  pa.pts_in = pts;
  pa.dout_in = dout;
  pa.time = time;
  return run_backward(s, net, pa, dgrid, dW, db, nullptr, st);
}

cudaError_t launch_fit_step(FitScratch& s, const NetDev& net, const FitArgs& a, cudaStream_t st) {
  if (!fit_supported(net)) return cudaErrorNotSupported;
  PointArgs pa{};
  pa.n = a.n;
  pa.mode = 0;
  pa.seed = a.seed;
  pa.step = a.step;
  pa.time = a.time;
  pa.vol = a.vol;
  pa.gw = a.grad_weight;
  pa.gs = a.grad_scale;
  pa.cdf = a.cdf;
  pa.cdf_res = a.cdf_res;
  pa.step_ptr = a.step_ptr;
  pa.stall_test = a.stall_test;
  const size_t ng = s.n_grid, nW = net_weight_count(net), nb = net_bias_count(net);
  cudaError_t e = run_backward(s, net, pa, s.grads, s.grads + ng, s.grads + ng + nW, a.loss, st, a.status);
  if (e != cudaSuccess) return e;
  const size_t n = ng + nW + nb;
  unsigned int blocks = (unsigned int)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 8);
  adam_kernel<<<blocks, 256, 0, st>>>(a.grid, a.weights, a.biases, s.grads, a.adam_m, a.adam_v, ng, nW, nb, a.lr_grid,
                                      a.lr_net, a.step, a.step_ptr, s.flag, a.status, a.grid_h, a.weights_h,
                                      a.grid_exp);
  return cudaGetLastError();
}

namespace {
__global__ void step_counter_kernel(int* step, int value, unsigned int* flag) {
  *step = value;
  *flag = 0u;
}
}  // namespace

cudaError_t launch_step_counter(int* step, int value, unsigned int* flag, cudaStream_t st) {
  step_counter_kernel<<<1, 1, 0, st>>>(step, value, flag);
  return cudaGetLastError();
}

}  // namespace srn
