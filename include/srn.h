/*
 * srn.h — C ABI of the GB300 (sm_103a) fV-SRN render / fit library.
 *
 * fV-SRN (Weiss, Hermüller, Westermann, "Fast Neural Representations for
 * Direct Volume Rendering", arXiv 2112.01579) represents a scalar volume by a
 * small MLP (Section 3) whose input is the position, its Fourier features
 * (Eq. 1-2) and a latent vector trilinearly interpolated from a dense latent
 * grid (Section 4.2).  This library evaluates that network at every sample
 * of a direct-volume-rendering ray march, trains it on density samples
 * (world-space L1 fit, Section 5 ablation setup), and computes its input
 * gradient for shading (Section 5 gradients).
 *
 * Conventions shared by every call
 * --------------------------------
 * - All array pointers named *_dev are CUDA device pointers owned by the
 *   caller; the library never frees them.  They must be 16-byte aligned.
 * - Pointers to structs (configs, cameras, transfer functions, descriptors)
 *   are host pointers; their contents are copied during the call.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued asynchronously on it; no call synchronizes
 *   except srn_sync_status, srn_save and srn_load.
 * - Arguments are validated before anything is enqueued: an invalid call
 *   returns SRN_ERR_INVALID_ARG or SRN_ERR_UNSUPPORTED with no side effect.
 *   A failed launch returns SRN_ERR_CUDA.  srn_last_error() gives the
 *   thread-local message of the last failure.
 * - There is no CPU fallback: every computation runs in the library's own
 *   CUDA kernels on the current device.
 *
 * Geometry
 * --------
 * The volume fills the world-space box [-0.5, 0.5]^3; network / volume
 * coordinates are p = x + 0.5 in [0, 1]^3.  Grids are vertex aligned: a grid
 * of n vertices per axis has vertex i at p = i / (n - 1) ("R vertices along
 * each axis", Section 4.2).  Volumes are float32 [nz][ny][nx] with x fastest.
 */
#ifndef SRN_H
#define SRN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum srn_status {
  SRN_OK = 0,
  SRN_ERR_INVALID_ARG = 1, /* a pointer, size or enum is invalid */
  SRN_ERR_UNSUPPORTED = 2, /* valid, but not a shape this build implements */
  SRN_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  SRN_ERR_NONFINITE = 4,   /* a fit step produced a non-finite loss/gradient */
  SRN_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  SRN_ERR_INTERNAL = 6     /* a device-side consistency check failed */
} srn_status;

enum { SRN_ACT_SINE = 0, SRN_ACT_SNAKEALT = 1 };   /* sin(x); Eq. 3: 0.5x + sin^2 x */
/* Network arithmetic of render / eval.  SRN_PREC_BF16 is named for
 * completeness and not implemented (srn_create returns SRN_ERR_UNSUPPORTED):
 * BF16 and FP16 run at the same tensor-core rate, BF16's 8-bit mantissa would
 * need the layer-0 inputs split into hi + lo as well (twice the operand tile
 * per warpgroup), and its wider range buys nothing the FP16 path lacks (the
 * latent grid is power-of-two scaled, hidden values beyond 65504 are outside
 * every FP32-accumulating kernel's tolerance). */
enum { SRN_PREC_FP32 = 0, SRN_PREC_FP16 = 1, SRN_PREC_BF16 = 2 };
enum { SRN_SHADE_NONE = 0, SRN_SHADE_ADJOINT = 1, SRN_SHADE_FD = 2, SRN_SHADE_HEAD = 3 };

#define SRN_MAX_KEYFRAMES 32
#define SRN_MAX_TF_POINTS 32
#define SRN_MAX_VIEWS 64
#define SRN_MAX_TIMES 64

/*
 * Network shape (Section 3 layer equation v_{i+1} = a(W_i v_i + b_i),
 * Section 4.1 m = (c-4)/2 rule, Section 4.2 latent grid, Section 7
 * keyframes).  Layer i maps d_i -> d_{i+1} with d_0 = 3 + 2m + F (input
 * [p, sin(Fp), cos(Fp), z]), d_1..d_{l-1} = width, d_l = out_dim; the
 * activation follows every layer but the last.
 */
typedef struct srn_config {
  int grid_res;    /* R >= 2: latent grid vertices per axis */
  int feat;        /* F: latent channels, a multiple of 4 (of 8 for FP16) */
  int n_fourier;   /* m: rows of the Fourier matrix */
  int layers;      /* l >= 2: number of linear layers */
  int width;       /* c: hidden channels: 32, 48 or 64 (the fused fit and backward: 32) */
  int out_dim;     /* D: 1 (density) or 4 (density + gradient head, Section 5) */
  int activation;  /* SRN_ACT_* */
  int precision;   /* SRN_PREC_*: arithmetic of srn_render (FP16 = tensor cores) */
  int n_keyframes; /* >= 1 latent grids; > 1 enables time interpolation */
  float key_times[SRN_MAX_KEYFRAMES]; /* increasing keyframe times (n_keyframes > 1) */
  int max_fit_points; /* scratch of srn_fit_step / srn_backward is sized for this many points (0: none) */
  int time_input;     /* 1: the time value is one more network input after z (Section 7 "direct"
                         encoding; d_0 = 3 + 2m + F + 1); 0: latent-only time interpolation */
  int grid_u8;        /* 1: the FP16 path reads an 8-bit latent grid (Section 4.2: per-channel
                         min/max mapped to [0,1], 8-bit codes) instead of grid_h */
} srn_config;

/*
 * Parameters, all device memory owned by the caller and read at call time
 * (updating them needs no re-create).  Layouts:
 *   grid     float32 [n_keyframes][R][R][R][F]   (x fastest, channel innermost)
 *   fourier  float32 [m][3]                      (fixed, not trained; Eq. 1)
 *   weights  float32 W_0 | W_1 | ... | W_{l-1}, each row-major [d_{i+1}][d_i]
 *   biases   float32 b_0 | ... | b_{l-1}
 *   grid_h / weights_h: FP16 copies with the same layouts, read by the FP16
 *            path; srn_sync_half writes them from the FP32 masters.
 *   adam_m / adam_v: float32 Adam moments packed [grid | weights | biases];
 *            required by srn_fit_step only.
 */
typedef struct srn_params {
  float* grid;
  const float* fourier;
  float* weights;
  float* biases;
  void* grid_h;
  void* weights_h;
  float* adam_m;
  float* adam_v;
  void* grid_q;    /* uint8 codes, layout of grid (grid_u8 only) */
  float* grid_qp;  /* float32 [F][2]: per-channel minimum and step (max - min) / 255 (grid_u8 only) */
} srn_params;

/* Pinhole camera: row 0 is the top row, rays through pixel centres. */
typedef struct srn_camera {
  float eye[3];
  float target[3];
  float up[3];
  float fovy; /* vertical field of view, radians */
} srn_camera;

/*
 * Transfer function (Section 3: densities are mapped to colour by a TF).
 * Density is clamped to [0,1]; RGBA is piecewise linear between the sorted
 * control points pos[0..n-1] (host arrays, copied), constant outside.
 * The extinction coefficient is A * opacity_scale per unit world length.
 */
typedef struct srn_tf {
  int n; /* 2..SRN_MAX_TF_POINTS */
  const float* pos;
  const float* rgba; /* n x 4 */
  float opacity_scale;
} srn_tf;

/*
 * Ray-march description.  Each ray is cut at the box into segments
 * [t0 + k step, min(t0 + (k+1) step, t1)], sampled at the segment midpoint,
 * alpha = 1 - exp(-kappa * length), composited front to back (premultiplied,
 * black background) and stopped after the sample that brings the opacity to
 * et_threshold or above (> 1 disables early termination).
 */
typedef struct srn_render_desc {
  int width, height;
  float step;         /* world units (the box is 1 wide) */
  float et_threshold; /* early ray termination opacity, e.g. 0.99 */
  int shading;        /* SRN_SHADE_*: headlight Blinn-Phong from the density gradient */
  float fd_h;         /* central-difference step (network coordinates) for SRN_SHADE_FD */
} srn_render_desc;

typedef struct srn_ctx srn_ctx;

/* Library version string (static storage). */
const char* srn_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char* srn_last_error(void);

/*
 * Create a context for one network.  Copies *cfg and *params (the pointed-to
 * device arrays are not copied and must outlive the context).  Allocates the
 * device scratch of the fit / backward (sized by cfg->max_fit_points) and a
 * small status word; nothing else allocates later.
 */
srn_status srn_create(const srn_config* cfg, const srn_params* params, srn_ctx** out);

/* Free the context's scratch.  Waits for the device first. */
srn_status srn_destroy(srn_ctx* ctx);

/* Replace the parameter pointers (same shapes). */
srn_status srn_set_params(srn_ctx* ctx, const srn_params* params);

/* Write grid_h / weights_h as the round-to-nearest FP16 of grid / weights;
 * with grid_u8, also the 8-bit grid: per channel f over all keyframes and
 * vertices, lo = min, step = (max - lo) / 255 (1 if max == lo), code =
 * round((g - lo) / step) clamped to [0, 255]; the network then sees
 * lo + step * code (Section 4.2 8-bit latent grid). */
srn_status srn_sync_half(srn_ctx* ctx, void* stream);

/*
 * fV-SRN direct volume rendering (the hot path): for every time in
 * times[0..n_times-1] (NULL: one frame at time 0) and every camera, render
 * an H x W image.  rgba_dev receives float32 [n_times][n_views][H][W][4],
 * premultiplied RGBA.  If samples_dev is not NULL the number of network
 * density samples taken is ADDED to *samples_dev (uint64).  Allocates
 * nothing (Section 6: fV-SRN decodes without temporary memory).
 * precision FP32: CUDA-core FP32; FP16: tensor-core MMA with FP32 accumulate.
 * FP16 operands hold magnitudes up to 65504: a network whose inputs or
 * activations exceed that renders non-finite densities, which the FP16 path
 * records as SRN_ERR_NONFINITE (reported by srn_sync_status); the FP32 path
 * evaluates such networks.
 */
srn_status srn_render(srn_ctx* ctx, const srn_camera* cams, int n_views, const float* times, int n_times,
                      const srn_tf* tf, const srn_render_desc* desc, float* rgba_dev,
                      unsigned long long* samples_dev, void* stream);

/*
 * Dense-grid DVR of a float32 volume (the plain method the network replaces;
 * Section 4 renders the original volume as the reference).  Same ray march,
 * density = trilinear interpolation of the volume; FD shading uses central
 * differences with a one-voxel step.  dims = {nx, ny, nz}, each >= 2.
 */
srn_status srn_dvr_dense(const float* volume_dev, const int dims[3], const srn_camera* cams, int n_views,
                         const srn_tf* tf, const srn_render_desc* desc, float* rgba_dev,
                         unsigned long long* samples_dev, void* stream);

/* Network output at n points (pts_dev float32 [n][3] in [0,1]^3) at one time:
 * out_dev float32 [n][D] (Section 3 network, Section 6 random-access decode).
 * Precision follows the context: FP32 CUDA cores, or the FP16 tensor-core
 * layers of the render (FP16 grid and weights, FP32 accumulate). */
srn_status srn_eval(srn_ctx* ctx, const float* pts_dev, int n, float time, float* out_dev, void* stream);

/* Density and its adjoint input gradient (Section 5 "Adjoint"): rho_dev [n],
 * grad_dev [n][3] (d rho / d p at the position clamped to [0,1]^3; may be
 * NULL).  Precision follows the context: FP32 CUDA cores, or on FP16 contexts
 * the tensor-core adjoint of the render (FP16 operands, hidden activations
 * and adjoint rows as FP16 hi + lo pairs, FP32 accumulate), which takes
 * networks of at most four layers, no time input, FP16 grid, of width 32
 * (12 Fourier rows / 8 latent channels or 14 / 16) or widths 48 / 64 (22 /
 * 30 Fourier rows, 16 latent channels, SnakeAlt); rho and the gradient are
 * those of output 0, so 4-output heads are taken too (other shapes on FP16
 * contexts: SRN_ERR_UNSUPPORTED). */
srn_status srn_density_grad(srn_ctx* ctx, const float* pts_dev, int n, float time, float* rho_dev,
                            float* grad_dev, void* stream);

/* Backward of srn_eval with respect to the positions (Section 5 "Adjoint",
 * seeded with dout): dpts_dev float32 [n][3] is OVERWRITTEN with
 * dpts_j = sum_d dout_j[d] d out_d / d p_j (derivative at the position
 * clamped to [0,1]^3), dout_dev float32 [n][D].  FP32 CUDA-core arithmetic
 * for every context precision (as srn_backward); allocates nothing. */
srn_status srn_input_backward(srn_ctx* ctx, const float* pts_dev, int n, float time, const float* dout_dev,
                              float* dpts_dev, void* stream);

/*
 * Parameter gradients of sum_j <dout_j, net(p_j)> (backward of srn_eval):
 * dgrid, dweights, dbiases are OVERWRITTEN (layouts of grid / weights /
 * biases).  dout_dev float32 [n][D].  n <= cfg.max_fit_points.  Deterministic:
 * the latent-grid gradient is gathered per vertex from points sorted by
 * cell, with no floating-point atomics.
 */
srn_status srn_backward(srn_ctx* ctx, const float* pts_dev, int n, float time, const float* dout_dev,
                        float* dgrid_dev, float* dweights_dev, float* dbiases_dev, void* stream);

/*
 * One training step (world-space fit): draw n_points positions with the
 * counter-based Philox4x32-10 generator keyed by (seed, step), take the
 * trilinear density of the volume there, L1 loss against the network output
 * (plus grad_weight * L1 of the head's gradient outputs against grad_scale
 * times central differences of the volume when D = 4), backpropagate, and
 * apply Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias correction at step+1)
 * with lr_grid on the latent grid and lr_net on weights and biases.  The
 * keyframe time of the samples is `time`.  Writes the loss (float32) to
 * loss_dev.  If the loss or any gradient is not finite the parameters are
 * left unchanged and the context records SRN_ERR_NONFINITE, reported by
 * srn_sync_status.  Also refreshes the FP16 copies when they exist.
 * Two-layer width-32 density networks (12 Fourier rows / 8 channels or
 * 14 / 16, no time input) run the per-point forward and the layer-0 weight
 * gradient on the tensor cores from FP16 hi + lo splits of FP32 values
 * (weight gradients within ~2e-4 of each block's maximum); every other shape
 * runs FP32 kernels.  Either way the step is deterministic.
 */
srn_status srn_fit_step(srn_ctx* ctx, const float* volume_dev, const int dims[3], int n_points, uint64_t seed,
                        int step, float time, float lr_grid, float lr_net, float grad_weight, float grad_scale,
                        float* loss_dev, void* stream);

/*
 * n_steps training steps first_step, first_step + 1, ... with the same
 * arguments: the same results, bit for bit, as that many srn_fit_step calls
 * (loss_dev holds the last step's loss), without the per-step launch cost.
 * One step is captured once as a CUDA graph on a stream the context owns
 * and replayed n_steps times on `stream`; the step index is kept in device
 * memory and advanced by the graph.  The graph is captured again when any
 * argument other than first_step / n_steps, the parameter arrays
 * (srn_set_params) or the adaptive distribution's storage changes (the
 * distribution's values are read at replay time).  n_steps >= 0 (0: nothing
 * happens), first_step >= 0, first_step + n_steps <= INT_MAX.  Validation and
 * error reporting as srn_fit_step; a non-finite step is skipped and
 * recorded, and the following steps run.
 */
srn_status srn_fit_steps(srn_ctx* ctx, const float* volume_dev, const int dims[3], int n_points, uint64_t seed,
                         int first_step, int n_steps, float time, float lr_grid, float lr_net, float grad_weight,
                         float grad_scale, float* loss_dev, void* stream);

/*
 * Section 6.2 adaptive resampling, step 1: the error grid.  err_dev
 * receives res^3 floats ([z][y][x], x fastest): E_v = mean over
 * samples_per_voxel positions in voxel v of |rho(p) - V(p)| (network output 0
 * in FP32 against the trilinear volume; paper: res 128, 8 positions).
 * Position i of voxel v = (vx, vy, vz): Philox4x32-10 of counter
 * (v, i, 0x4552, 0), key (seed low, seed high); u_a = (word_a >> 8) 2^-24;
 * p_a = (v_a + u_a) / res in FP32 round-to-nearest.  2 <= res <= 256,
 * 1 <= samples_per_voxel <= 64.  Any width.
 */
srn_status srn_error_grid(srn_ctx* ctx, const float* volume_dev, const int dims[3], int res, int samples_per_voxel,
                          uint64_t seed, float time, float* err_dev, void* stream);

/*
 * Section 6.2 adaptive resampling, step 2: later srn_fit_step calls draw
 * their points with counts proportional to the error grid err_dev (res^3
 * floats, e.g. from srn_error_grid; read now, not kept).  Weights
 * q_v = floor(E_v * (65535 / max E)) in FP32; S = exclusive prefix sum of q
 * (64-bit integers), Q = S[res^3].  Point j of n lies in the voxel v with
 * S[v] <= floor((2j + 1) Q / (2n)) < S[v + 1] (voxel v receives
 * round(n q_v / Q) points, +-1), at the offset the uniform sampler's Philox
 * draw for (seed, step, j) gives inside the voxel: p_a = (v_a + u_a) / res as
 * above.  err_dev = NULL, or a grid whose maximum is 0, returns to uniform
 * sampling.  A negative or non-finite entry leaves the sampling unchanged and
 * returns SRN_ERR_INVALID_ARG (the call synchronizes the stream to check).
 * The distribution lives in context memory (allocated on the first call or
 * when res grows).  2 <= res <= 256.
 */
srn_status srn_fit_set_sampling(srn_ctx* ctx, const float* err_dev, int res, void* stream);

/* The n_points positions (float32 [n][3]) that srn_fit_step with the same
 * (n_points, seed, step) draws under the current sampling (uniform or
 * adaptive). */
srn_status srn_fit_points(srn_ctx* ctx, int n_points, uint64_t seed, int step, float* pts_dev, void* stream);

/* Mean squared difference of two float32 arrays of n values (densities):
 * PSNR = 10 log10(1 / MSE) for volumes normalised to [0,1] (Section 6
 * reports reconstruction PSNR).  One double to mse_dev; deterministic (a
 * fixed two-level FP64 reduction over all SMs whose 8 KB of partial sums
 * are stream-ordered scratch: cudaMallocAsync / cudaFreeAsync on `stream`). */
srn_status srn_density_mse(const float* a_dev, const float* b_dev, long long n, double* mse_dev, void* stream);

/* Vertex-aligned trilinear resampling of a float32 volume src_dims = {nx,
 * ny, nz} onto a grid of dst_dims (each >= 1; a 1-vertex axis samples p = 0). */
srn_status srn_resample(const float* src_dev, const int src_dims[3], float* dst_dev, const int dst_dims[3],
                        void* stream);

/*
 * The "off" baseline of Section 6.2: the volume low-pass filtered and
 * downsampled to an M^3 density grid of the latent grid's memory
 * (M = round(cbrt(R^3 F)), e.g. 81 for 32^3 x 16).  Separable Gaussian with
 * sigma = 0.5 (n_a - 1) / (M - 1) voxels per axis, truncated at 3 sigma,
 * clamp-to-edge, then vertex-aligned trilinear resampling.  tmp_dev holds
 * 2 nx ny nz floats; out_dev receives M^3 floats.
 */
srn_status srn_lowpass_resample(const float* volume_dev, const int dims[3], int M, float* tmp_dev, float* out_dev,
                                void* stream);

/*
 * srn_backward for callers that cannot allocate device memory.  The paper
 * has no counterpart; this exists for integrators, not for the method.
 *
 * Some callers must not call cudaMalloc: hosts whose device memory is
 * owned by another allocator (a framework's caching pool, or an arena sized
 * once at start-up whose budget an outside allocation would break), and
 * frame loops that may not take the device-wide synchronization that
 * cudaMalloc / cudaFree can cause.  srn_create allocates scratch, so such
 * callers cannot use srn_backward; this entry point needs no context and
 * allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 *
 * It computes exactly what srn_backward computes for the network described
 * by *cfg / *params (same arguments, same outputs, overwritten), using a
 * fixed device scratch area of SRN_STATIC_SCRATCH_BYTES that every GPU
 * loading the library holds until the process exits.  Limits and rules:
 * - n is limited by that area; the largest n depends on the network shape
 *   (about 260k points for an 8^3 x 8 grid, about 150k for 32^3 x 16).  A
 *   larger n returns SRN_ERR_INVALID_ARG and srn_last_error() states the
 *   largest n that fits.  cfg->max_fit_points is ignored.
 * - The first call on each device looks up the area's device address
 *   (once per device, with that device current) and keeps it for the life
 *   of the process; make that first call before any stream capture begins.
 *   The kept address is not valid after cudaDeviceReset on that device, so
 *   do not use this entry point in a process that resets the device.
 * - n = 0 is valid and writes zeros to every output.
 * - All calls share the one area, which keeps the previous call's contents
 *   (everything the call relies on is rewritten first).  Calls whose work
 *   overlaps on the GPU (different streams, or different host threads) race
 *   on it: serialize them.
 */
#define SRN_STATIC_SCRATCH_BYTES (16u << 20)
srn_status srn_backward_static(const srn_config* cfg, const srn_params* params, const float* pts_dev, int n,
                               float time, const float* dout_dev, float* dgrid_dev, float* dweights_dev,
                               float* dbiases_dev, void* stream);

/*
 * Checkpoint of a context's network: the shape fields of its config, the
 * FP32 grid, weights and biases, the Adam moments when the context has them,
 * and the caller's step counter (the fit's sampler and bias correction are
 * keyed by it, so a resumed fit reproduces the uninterrupted one exactly).
 * Little-endian binary file with a magic, a version and counts.  Both calls
 * synchronize the device.  srn_load requires a context of the same shape
 * (SRN_ERR_INVALID_ARG otherwise), writes into the context's parameter
 * arrays, refreshes the FP16 copies and returns the step in *step_out.
 */
srn_status srn_save(srn_ctx* ctx, const char* path, int step);
srn_status srn_load(srn_ctx* ctx, const char* path, int* step_out);

/* Synchronize `stream` and return (then clear) the device status word:
 * SRN_OK, SRN_ERR_NONFINITE, SRN_ERR_TIMEOUT or SRN_ERR_INTERNAL.
 * SRN_ERR_TIMEOUT: a bounded wait of the tensor-core kernels (about one
 * second of clock) ran out; the kernel left its loop, freed its tensor
 * memory and returned, and the context stays usable (a fit step that timed
 * out leaves parameters and Adam moments as they were).  For testing that
 * path, srn_render and srn_fit_step(s) read the environment variable
 * SRN_TEST_STALL at each call: when it is "1" the tensor-core render and the
 * tensor-core fit point kernel issue no MMA, so every wait runs out. */
srn_status srn_sync_status(srn_ctx* ctx, void* stream);

/* Mean squared error over the RGB channels of n RGBA float32 pixels, the
 * quantity behind the PSNR = 10 log10(1 / MSE) the paper reports for image
 * quality (Section 6).  Writes one double to mse_dev; deterministic, with
 * the reduction and scratch of srn_density_mse. */
srn_status srn_image_mse(const float* a_dev, const float* b_dev, long long n_pixels, double* mse_dev,
                         void* stream);

/* Structural similarity (Wang, Bovik, Sheikh, Simoncelli 2004) of two
 * height x width RGBA float32 images ([y][x][4], 16-byte aligned; alpha
 * ignored), the second image-quality measure the evaluation states beside
 * PSNR (Section 6): 11 x 11 Gaussian window of sigma 1.5 normalised to sum
 * 1, K1 = 0.01, K2 = 0.03, dynamic range 1; the mean over the R, G, B
 * channels and every window centre whose window lies inside the image
 * (1.0 when none does).  Computed in FP64; one double to ssim_dev;
 * deterministic (fixed tiles, fixed-order sums; stream-ordered scratch of
 * one double per 32 x 8 tile of window centres).  width, height >= 1. */
srn_status srn_image_ssim(const float* a_dev, const float* b_dev, int width, int height, double* ssim_dev,
                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SRN_H */
