// Internal interface of the fit / backward kernels (world-space training).
#pragma once

#include "srn_internal.h"

namespace srn {

// Device scratch owned by a context, sized for max_fit_points points.
struct FitScratch {
  int max_points;
  int n_blocks;              // CTAs of the per-point kernel
  float* pts;                // [n][3] sampled positions
  float* target;             // [n] ground-truth density (and [n][3] gradient targets for D = 4)
  float* dout;               // [n][D] output adjoints
  float* dz;                 // [n][F] latent adjoints (times keyframe weight applied later)
  unsigned int* key;         // [n] cell index of each point
  unsigned int* key_alt;     // [n] radix-sort ping-pong
  unsigned int* idx;         // [n] point index, sorted by cell
  unsigned int* idx_alt;     // [n]
  unsigned int* hist;        // radix histogram [256][n_sort_blocks]
  unsigned int* cell_start;  // [n_cells + 1]
  float* dW_part;            // [n_blocks][n_weights + n_biases] per-CTA partial sums
  float* loss_part;          // [n_blocks] per-CTA loss partials
  float* grads;              // [grid | W | b] full gradient of one step
  float* cell_part;          // [n_cells][8][F] per-cell corner partials
  size_t n_cells;
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
  float* adam_m;
  float* adam_v;
};

cudaError_t fit_scratch_alloc(FitScratch& s, const NetDev& net, int max_points);
void fit_scratch_free(FitScratch& s);
cudaError_t launch_backward(FitScratch& s, const NetDev& net, const float* pts, int n, float time, const float* dout,
                            float* dgrid, float* dW, float* db, cudaStream_t st);
cudaError_t launch_fit_step(FitScratch& s, const NetDev& net, const FitArgs& a, cudaStream_t st);

}  // namespace srn
