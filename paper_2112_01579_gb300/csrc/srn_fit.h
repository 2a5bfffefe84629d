// Internal interface of the fit / backward kernels (world-space training).
#pragma once

#include "srn_internal.h"

namespace srn {

// Device scratch owned by a context, sized for max_points points.
struct FitScratch {
  int max_points;
  int max_cta;             // CTAs of the per-point kernel (partials rows)
  size_t n_cells;          // (R-1)^3 latent-grid cells
  size_t n_entries;        // weights + biases
  size_t n_grid;           // latent-grid entries over all keyframes
  int radix_bins;          // 256 (8-bit digits) or 512 (one 9-bit pass for up to 512 cells)
  float* pts;              // [n][3] positions (clamped) of the current step
  float* dz;               // [n][F] adjoint of the latent vector
  unsigned int* key;       // [n] cell of each point, and radix ping-pong
  unsigned int* key_alt;
  unsigned int* idx;       // [n] point index, sorted by cell
  unsigned int* idx_alt;
  unsigned int* hist;      // radix histograms [256][sort blocks]
  unsigned int* digit_totals;  // [radix_bins] keys per digit in one sort pass
  unsigned int* cell_start;  // [n_cells + 1]
  float* part;             // [max_cta][n_entries + 1] per-CTA weight-gradient / loss partials
  float* grads;            // [n_grid + n_entries] gradient of one step (grid | weights | biases)
  unsigned int* flag;      // non-finite flag of the current step
  float* cell_part;        // [n_cells][8][F] per-(cell, corner) partials (small grids; may be null)
};

struct FitArgs {
  VolDev vol;
  int n;
  unsigned long long seed;
  int step;
  float time;
  float lr_grid, lr_net, grad_weight, grad_scale;
  float* loss;
  unsigned int* status;
  float* grid;
  float* weights;
  float* biases;
  __half* grid_h;
  __half* weights_h;
  const int* grid_exp;  // FP16 grid scale exponent: grid_h = fp16(grid 2^-k) (see NetDev)
  float* adam_m;
  float* adam_v;
  const unsigned long long* cdf;  // Section 6.2 adaptive distribution over cdf_res^3 voxels (null: uniform)
  int cdf_res;
  int* step_ptr;  // when not null, the step index is read from here (CUDA-graph replay), not `step`, and
                  // the step's last kernel (Adam) advances it by one
  int stall_test;  // test of the timeout path: the tensor-core point kernel issues no MMA
};

bool fit_supported(const NetDev& net);
// Radix bins of the cell sort: 512 (one 9-bit pass) for up to 512 cells, else 256.
int sort_bins(size_t n_cells);
cudaError_t fit_scratch_alloc(FitScratch& s, const NetDev& net, int max_points);
void fit_scratch_free(FitScratch& s);
cudaError_t launch_backward(FitScratch& s, const NetDev& net, const float* pts, int n, float time, const float* dout,
                            float* dgrid, float* dW, float* db, cudaStream_t st);
cudaError_t launch_fit_step(FitScratch& s, const NetDev& net, const FitArgs& a, cudaStream_t st);
// *step = value and the scratch's non-finite flag cleared, one thread (before
// the first step of a graph-replayed run).
cudaError_t launch_step_counter(int* step, int value, unsigned int* flag, cudaStream_t st);

// Tensor-core point kernel of the fit (srn_fit_mma.cu): arguments, support
// (width 32, two layers, density output, no time input, 12 Fourier rows / 8
// channels or 14 / 16), partial rows written per CTA.
struct PointArgsMma {
  int n;
  unsigned long long seed;
  int step;
  float time;
  VolDev vol;
  const unsigned long long* cdf;
  int cdf_res;
  const int* step_ptr;  // when not null, the step index (overrides `step`)
  float* pts;
  float* dz;
  unsigned int* key;
  unsigned int* idx;
  float* part;
  unsigned int* flag;  // bit 1: a bounded wait gave up (the step's Adam then skips the update)
  int stall_test;      // test of the timeout path: issue no MMA, so every wait runs out
};
bool fit_mma_supported(const NetDev& n);
int fit_mma_rows_per_cta();
cudaError_t launch_fit_mma(const NetDev& n, const PointArgsMma& a, int grid, unsigned int* status, cudaStream_t st);

// Section 6.2 adaptive resampling (srn_adaptive.cu).
// Error grid E[res^3]: mean |net(p) - V(p)| over spv positions per voxel.
cudaError_t launch_error_grid(const NetDev& net, const VolDev& vol, int res, int spv, unsigned long long seed,
                              float time, float* E, cudaStream_t st);
// Validity and maximum of E: flags[0] = 1 if an entry is negative or not
// finite, flags[1] = bits of the maximum (E >= 0 orders like its bits).
cudaError_t launch_error_max(const float* E, long long n, unsigned int* flags, cudaStream_t st);
// Integer distribution S[n + 1] (exclusive prefix of the 16-bit weights)
// from E and its maximum in flags[1]; bsum holds ceil(n / 2048) entries.
cudaError_t launch_build_cdf(const float* E, long long n, const unsigned int* flags, unsigned long long* S,
                             unsigned long long* bsum, cudaStream_t st);
// The n points a fit step (seed, step) draws under S (null: uniform).
cudaError_t launch_fit_points(const unsigned long long* S, int res, unsigned long long seed, int step, int n,
                              float* pts, cudaStream_t st);
constexpr int kCdfBlock = 2048;  // weights per block of the prefix sum

}  // namespace srn
