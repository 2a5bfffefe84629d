// C ABI of the library (include/srn.h): argument validation, context
// management and kernel dispatch.  No computation happens here: every step
// of the render / eval / fit path runs in the library's CUDA kernels.
#include <limits.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>

#include "srn_fit.h"
#include "srn_internal.h"

using namespace srn;

struct srn_ctx {
  srn_config cfg;
  srn_params prm;
  int device;
  // device words: [0] status (SRN_OK / SRN_ERR_NONFINITE / ...), [1] graph step
  // index, [2..3] render work counter, [4] FP16 latent-grid scale exponent,
  // [5] scratch of its computation (bits of max |grid|)
  unsigned int* status;
  unsigned long long* ray_counter;  // persistent-render work counter (8-byte aligned)
  FitScratch fit;             // scratch of srn_fit_step / srn_backward
  // Section 6.2 adaptive distribution (srn_fit_set_sampling)
  unsigned long long* cdf = nullptr;   // [cdf_cap] exclusive prefix sums of the voxel weights
  unsigned long long* cdf_bsum = nullptr;
  unsigned int* cdf_flags = nullptr;   // [2] validity flag, maximum bits
  size_t cdf_cap = 0;
  int cdf_res = 0;
  bool cdf_active = false;
  // srn_fit_steps: one fit step captured as a CUDA graph, replayed per step;
  // the step index lives in status[1] and the graph advances it.
  cudaStream_t graph_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  srn::FitArgs graph_key;  // the arguments baked into graph_exec
};

namespace {

thread_local char g_err[512] = "";

srn_status fail(srn_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

srn_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SRN_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Host-side switch for testing the timeout path: with SRN_TEST_STALL=1 in the
// environment, srn_render and the fit's tensor-core point kernel issue no MMA,
// so their bounded mbarrier waits run out (~1 s of clock) and report
// SRN_ERR_TIMEOUT; a fit step then leaves the parameters as they are.
bool test_stall() {
  const char* v = getenv("SRN_TEST_STALL");
  return v && v[0] == '1' && v[1] == 0;
}

// (2n + 1) * Q < 2^64 for every adaptive distribution over res^3 voxels
// (Q <= 65535 res^3), so the stratum midpoints stay exact in 64 bits.
bool adaptive_fits(long long n, int res) {
  const unsigned long long q = 65535ull * (unsigned)res * (unsigned)res * (unsigned)res;
  return q <= ~0ull / (2ull * (unsigned long long)n + 1ull);
}

srn_status check_config(const srn_config* c) {
  if (!c) return fail(SRN_ERR_INVALID_ARG, "config is NULL");
  if (c->grid_res < 2) return fail(SRN_ERR_INVALID_ARG, "grid_res must be >= 2");
  if (c->feat < 4 || c->feat % 4) return fail(SRN_ERR_INVALID_ARG, "feat must be a positive multiple of 4");
  if (c->n_fourier < 0) return fail(SRN_ERR_INVALID_ARG, "n_fourier must be >= 0");
  if (c->layers < 2) return fail(SRN_ERR_INVALID_ARG, "layers must be >= 2");
  if (c->layers > 8) return fail(SRN_ERR_UNSUPPORTED, "at most 8 layers are implemented");
  if (c->out_dim != 1 && c->out_dim != 4) return fail(SRN_ERR_INVALID_ARG, "out_dim must be 1 or 4");
  if (c->activation != SRN_ACT_SINE && c->activation != SRN_ACT_SNAKEALT)
    return fail(SRN_ERR_INVALID_ARG, "unknown activation");
  if (c->precision == SRN_PREC_BF16)
    return fail(SRN_ERR_UNSUPPORTED, "BF16 network arithmetic is not implemented (FP16 tensor cores or FP32)");
  if (c->precision != SRN_PREC_FP32 && c->precision != SRN_PREC_FP16)
    return fail(SRN_ERR_INVALID_ARG, "unknown precision");
  if (c->n_keyframes < 1 || c->n_keyframes > SRN_MAX_KEYFRAMES)
    return fail(SRN_ERR_INVALID_ARG, "n_keyframes must be in [1, %d]", SRN_MAX_KEYFRAMES);
  for (int k = 1; k < c->n_keyframes; ++k)
    if (!(c->key_times[k] > c->key_times[k - 1])) return fail(SRN_ERR_INVALID_ARG, "key_times must increase");
  if (c->max_fit_points < 0) return fail(SRN_ERR_INVALID_ARG, "max_fit_points must be >= 0");
  if (!render_fp32_supported(c->width)) return fail(SRN_ERR_UNSUPPORTED, "width %d is not implemented", c->width);
  if (c->time_input != 0 && c->time_input != 1) return fail(SRN_ERR_INVALID_ARG, "time_input must be 0 or 1");
  if (c->grid_u8 != 0 && c->grid_u8 != 1) return fail(SRN_ERR_INVALID_ARG, "grid_u8 must be 0 or 1");
  if (c->grid_u8 && c->precision != SRN_PREC_FP16)
    return fail(SRN_ERR_INVALID_ARG, "the 8-bit grid is read by the FP16 path only");
  if (3 + 2 * c->n_fourier + c->feat + c->time_input > 256)
    return fail(SRN_ERR_UNSUPPORTED, "network input wider than 256");
  if ((size_t)c->grid_res * c->grid_res * c->grid_res * c->feat * c->n_keyframes > (size_t)1 << 31)
    return fail(SRN_ERR_UNSUPPORTED, "latent grid larger than 2^31 entries");
  return SRN_OK;
}

srn_status check_params(const srn_config* c, const srn_params* p) {
  if (!p) return fail(SRN_ERR_INVALID_ARG, "params is NULL");
  if (!p->grid || !p->weights || !p->biases || (c->n_fourier > 0 && !p->fourier))
    return fail(SRN_ERR_INVALID_ARG, "grid, weights, biases and fourier are required");
  if (!aligned16(p->grid) || !aligned16(p->grid_h) || !aligned16(p->weights))
    return fail(SRN_ERR_INVALID_ARG, "parameter arrays must be 16-byte aligned");
  if (c->precision == SRN_PREC_FP16 && (!p->grid_h || !p->weights_h))
    return fail(SRN_ERR_INVALID_ARG, "FP16 precision needs grid_h and weights_h");
  if (c->grid_u8 && (!p->grid_q || !p->grid_qp || !aligned16(p->grid_q)))
    return fail(SRN_ERR_INVALID_ARG, "the 8-bit grid needs 16-byte aligned grid_q and grid_qp");
  return SRN_OK;
}

NetDev make_net(const srn_ctx* ctx) {
  NetDev n;
  const srn_config& c = ctx->cfg;
  n.grid = ctx->prm.grid;
  n.grid_h = reinterpret_cast<const __half*>(ctx->prm.grid_h);
  n.fourier = ctx->prm.fourier;
  n.W = ctx->prm.weights;
  n.W_h = reinterpret_cast<const __half*>(ctx->prm.weights_h);
  n.b = ctx->prm.biases;
  n.R = c.grid_res; n.F = c.feat; n.m = c.n_fourier; n.l = c.layers; n.c = c.width; n.D = c.out_dim;
  n.act = c.activation; n.nkey = c.n_keyframes; n.ti = c.time_input;
  n.gq = c.grid_u8;
  n.grid_q = reinterpret_cast<const uint8_t*>(ctx->prm.grid_q);
  n.grid_qp = ctx->prm.grid_qp;
  n.grid_exp = ctx->status ? reinterpret_cast<const int*>(ctx->status + 4) : nullptr;
  for (int k = 0; k < SRN_MAX_KEYFRAMES; ++k) n.key_times[k] = k < c.n_keyframes ? c.key_times[k] : 0.0f;
  return n;
}

// FP16 copies of the FP32 masters: the latent grid with its power-of-two
// scale (exponent into status[4]), the weights as they are, the 8-bit grid.
cudaError_t write_half_copies(srn_ctx* ctx, cudaStream_t s) {
  const NetDev n = make_net(ctx);
  cudaError_t e = launch_grid_to_half_scaled(n.grid, (__half*)ctx->prm.grid_h, net_grid_count(n),
                                             reinterpret_cast<int*>(ctx->status + 4), s);
  if (e == cudaSuccess) e = launch_to_half(n.W, (__half*)ctx->prm.weights_h, net_weight_count(n), s);
  if (e == cudaSuccess && ctx->cfg.grid_u8)
    e = launch_quantize_grid(n.grid, net_grid_count(n) / n.F, n.F, (uint8_t*)ctx->prm.grid_q, ctx->prm.grid_qp, s);
  return e;
}

// Camera frame in FP64 (view set-up, once per camera and call), stored as
// FP32 pairs hi + lo; see CamDev.
void split2(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

CamDev camera_frame(const srn_camera& c, int W, int H) {
  double f[3], r[3], u[3];
  for (int a = 0; a < 3; ++a) f[a] = (double)c.target[a] - (double)c.eye[a];
  const double nf = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (int a = 0; a < 3; ++a) f[a] /= nf;
  const double up[3] = {c.up[0], c.up[1], c.up[2]};
  r[0] = f[1] * up[2] - f[2] * up[1];
  r[1] = f[2] * up[0] - f[0] * up[2];
  r[2] = f[0] * up[1] - f[1] * up[0];
  const double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int a = 0; a < 3; ++a) r[a] /= nr;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  const double th = tan(0.5 * (double)c.fovy);
  CamDev d;
  for (int a = 0; a < 3; ++a) {
    d.eye[a] = c.eye[a];
    split2(f[a], d.f[a], d.fl[a]);
    split2(r[a], d.r[a], d.rl[a]);
    split2(u[a], d.u[a], d.ul[a]);
  }
  split2(th, d.th[0], d.th[1]);
  split2(th * ((double)W / (double)H), d.tha[0], d.tha[1]);
  return d;
}

srn_status fill_batch(BatchDev& b, const srn_camera* cams, int n_views, const float* times, int n_times,
                      const srn_tf* tf, const srn_render_desc* desc, float* rgba, unsigned long long* samples,
                      bool network) {
  memset(&b, 0, sizeof(b));
  if (!cams || n_views < 1 || n_views > SRN_MAX_VIEWS)
    return fail(SRN_ERR_INVALID_ARG, "need 1..%d cameras", SRN_MAX_VIEWS);
  if (n_times < 1 || n_times > SRN_MAX_TIMES) return fail(SRN_ERR_INVALID_ARG, "need 1..%d times", SRN_MAX_TIMES);
  if (times == nullptr && n_times != 1) return fail(SRN_ERR_INVALID_ARG, "times is NULL but n_times != 1");
  if (!tf || tf->n < 2 || tf->n > SRN_MAX_TF_POINTS || !tf->pos || !tf->rgba)
    return fail(SRN_ERR_INVALID_ARG, "transfer function needs 2..%d points", SRN_MAX_TF_POINTS);
  for (int i = 1; i < tf->n; ++i)
    if (!(tf->pos[i] >= tf->pos[i - 1])) return fail(SRN_ERR_INVALID_ARG, "TF control points must be sorted");
  if (!(tf->opacity_scale >= 0.0f) || !isfinite(tf->opacity_scale))
    return fail(SRN_ERR_INVALID_ARG, "opacity_scale must be finite and >= 0");
  if (!desc || desc->width < 1 || desc->height < 1) return fail(SRN_ERR_INVALID_ARG, "bad image size");
  if (!(desc->step >= 1e-5f) || !isfinite(desc->step)) return fail(SRN_ERR_INVALID_ARG, "step must be >= 1e-5");
  if (desc->shading < SRN_SHADE_NONE || desc->shading > SRN_SHADE_HEAD)
    return fail(SRN_ERR_INVALID_ARG, "unknown shading mode");
  if (network && desc->shading == SRN_SHADE_FD && !(desc->fd_h > 0.0f)) return fail(SRN_ERR_INVALID_ARG, "fd_h must be > 0");
  if (!rgba || !aligned16(rgba)) return fail(SRN_ERR_INVALID_ARG, "rgba_dev must be a 16-byte aligned pointer");
  if ((long long)desc->width * desc->height * n_views * n_times > (1ll << 34))
    return fail(SRN_ERR_UNSUPPORTED, "batch too large");
  for (int v = 0; v < n_views; ++v) {
    const srn_camera& c = cams[v];
    float f[3] = {c.target[0] - c.eye[0], c.target[1] - c.eye[1], c.target[2] - c.eye[2]};
    float r[3] = {f[1] * c.up[2] - f[2] * c.up[1], f[2] * c.up[0] - f[0] * c.up[2], f[0] * c.up[1] - f[1] * c.up[0]};
    if (f[0] * f[0] + f[1] * f[1] + f[2] * f[2] == 0.0f || r[0] * r[0] + r[1] * r[1] + r[2] * r[2] == 0.0f ||
        !(c.fovy > 0.0f && c.fovy < 3.14159f))
      return fail(SRN_ERR_INVALID_ARG, "camera %d is degenerate", v);
    b.cams[v] = camera_frame(c, desc->width, desc->height);
  }
  for (int t = 0; t < n_times; ++t) b.times[t] = times ? times[t] : 0.0f;
  b.n_views = n_views;
  b.n_times = n_times;
  b.W = desc->width;
  b.H = desc->height;
  b.step = desc->step;
  b.et = desc->et_threshold;
  b.shading = desc->shading;
  b.fd_h = desc->fd_h;
  b.tf.n = tf->n;
  b.tf.opacity_scale = tf->opacity_scale;
  for (int i = 0; i < SRN_MAX_TF_POINTS; ++i) {
    int k = i < tf->n ? i : tf->n - 1;
    b.tf.pos[i] = tf->pos[k];
    b.tf.rgba[i] = make_float4(tf->rgba[4 * k], tf->rgba[4 * k + 1], tf->rgba[4 * k + 2], tf->rgba[4 * k + 3]);
  }
  b.out = rgba;
  b.samples = samples;
  return SRN_OK;
}

srn_status use_device(const srn_ctx* ctx) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != ctx->device) return fail(SRN_ERR_INVALID_ARG, "context belongs to device %d, current is %d", ctx->device, cur);
  return SRN_OK;
}

}  // namespace

extern "C" {

const char* srn_version(void) { return "fvsrn-gb300 0.1 (sm_103a)"; }

const char* srn_last_error(void) { return g_err; }

srn_status srn_create(const srn_config* cfg, const srn_params* params, srn_ctx** out) {
  if (!out) return fail(SRN_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  srn_status st = check_config(cfg);
  if (st) return st;
  st = check_params(cfg, params);
  if (st) return st;
  srn_ctx* ctx = new (std::nothrow) srn_ctx;
  if (!ctx) return fail(SRN_ERR_INTERNAL, "out of host memory");
  memset(ctx, 0, sizeof(*ctx));
  ctx->cfg = *cfg;
  ctx->prm = *params;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->status, 8 * sizeof(unsigned int));
  if (e == cudaSuccess) {
    ctx->ray_counter = reinterpret_cast<unsigned long long*>(ctx->status + 2);
    e = cudaMemset(ctx->status, 0, 8 * sizeof(unsigned int));
  }
  if (e == cudaSuccess) e = fit_scratch_alloc(ctx->fit, make_net(ctx), cfg->max_fit_points);
  if (e != cudaSuccess) {
    fit_scratch_free(ctx->fit);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
    return cuda_fail(e, "srn_create");
  }
  *out = ctx;
  return SRN_OK;
}

srn_status srn_destroy(srn_ctx* ctx) {
  if (!ctx) return SRN_OK;
  cudaDeviceSynchronize();
  fit_scratch_free(ctx->fit);
  if (ctx->cdf) cudaFree(ctx->cdf);
  if (ctx->cdf_bsum) cudaFree(ctx->cdf_bsum);
  if (ctx->cdf_flags) cudaFree(ctx->cdf_flags);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph_stream) cudaStreamDestroy(ctx->graph_stream);
  if (ctx->status) cudaFree(ctx->status);
  delete ctx;
  return SRN_OK;
}

srn_status srn_set_params(srn_ctx* ctx, const srn_params* params) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  srn_status st = check_params(&ctx->cfg, params);
  if (st) return st;
  ctx->prm = *params;
  return SRN_OK;
}

srn_status srn_sync_half(srn_ctx* ctx, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->prm.grid_h || !ctx->prm.weights_h) return fail(SRN_ERR_INVALID_ARG, "no FP16 copies to write");
  srn_status st = use_device(ctx);
  if (st) return st;
  cudaError_t e = write_half_copies(ctx, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_sync_half");
}

srn_status srn_render(srn_ctx* ctx, const srn_camera* cams, int n_views, const float* times, int n_times,
                      const srn_tf* tf, const srn_render_desc* desc, float* rgba_dev,
                      unsigned long long* samples_dev, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  BatchDev b;
  srn_status st = fill_batch(b, cams, n_views, times, n_times, tf, desc, rgba_dev, samples_dev, true);
  if (st) return st;
  b.stall_test = test_stall();
  if (desc->shading == SRN_SHADE_HEAD && ctx->cfg.out_dim != 4)
    return fail(SRN_ERR_INVALID_ARG, "head shading needs out_dim 4");
  st = use_device(ctx);
  if (st) return st;
  NetDev n = make_net(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (ctx->cfg.precision == SRN_PREC_FP16) {
    if (!render_mma_supported(n, desc->shading))
      return fail(SRN_ERR_UNSUPPORTED, "FP16 tensor-core render does not implement this shape / shading");
    e = launch_render_mma(n, b, ctx->ray_counter, ctx->status, s);
  } else {
    e = launch_render_fp32(n, b, s);
  }
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_render");
}

srn_status srn_dvr_dense(const float* volume_dev, const int dims[3], const srn_camera* cams, int n_views,
                         const srn_tf* tf, const srn_render_desc* desc, float* rgba_dev,
                         unsigned long long* samples_dev, void* stream) {
  if (!volume_dev || !dims) return fail(SRN_ERR_INVALID_ARG, "volume and dims are required");
  if (dims[0] < 2 || dims[1] < 2 || dims[2] < 2) return fail(SRN_ERR_INVALID_ARG, "volume dims must be >= 2");
  BatchDev b;
  srn_status st = fill_batch(b, cams, n_views, nullptr, 1, tf, desc, rgba_dev, samples_dev, false);
  if (st) return st;
  if (desc->shading != SRN_SHADE_NONE && desc->shading != SRN_SHADE_FD)
    return fail(SRN_ERR_INVALID_ARG, "dense DVR shades by central differences only");
  VolDev v{volume_dev, dims[0], dims[1], dims[2]};
  cudaError_t e = launch_dvr_dense(v, b, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_dvr_dense");
}

srn_status srn_eval(srn_ctx* ctx, const float* pts_dev, int n, float time, float* out_dev, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || (n > 0 && (!pts_dev || !out_dev))) return fail(SRN_ERR_INVALID_ARG, "bad points / output");
  srn_status st = use_device(ctx);
  if (st) return st;
  const NetDev net = make_net(ctx);
  cudaError_t e;
  if (ctx->cfg.precision == SRN_PREC_FP16) {
    if (!eval_mma_supported(net)) return fail(SRN_ERR_UNSUPPORTED, "FP16 tensor-core eval does not implement this shape");
    e = launch_eval_mma(net, pts_dev, n, time, out_dev, ctx->ray_counter, ctx->status, (cudaStream_t)stream);
  } else {
    e = launch_eval_fp32(net, pts_dev, n, time, out_dev, nullptr, 0, (cudaStream_t)stream);
  }
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_eval");
}

srn_status srn_density_grad(srn_ctx* ctx, const float* pts_dev, int n, float time, float* rho_dev,
                            float* grad_dev, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || (n > 0 && (!pts_dev || !rho_dev))) return fail(SRN_ERR_INVALID_ARG, "bad points / output");
  srn_status st = use_device(ctx);
  if (st) return st;
  const NetDev net = make_net(ctx);
  cudaError_t e;
  if (ctx->cfg.precision == SRN_PREC_FP16) {
    if (!density_grad_mma_supported(net))
      return fail(SRN_ERR_UNSUPPORTED, "the FP16 tensor-core adjoint does not implement this shape");
    e = launch_density_grad_mma(net, pts_dev, n, time, rho_dev, grad_dev, ctx->ray_counter, ctx->status,
                                (cudaStream_t)stream);
  } else {
    e = launch_eval_fp32(net, pts_dev, n, time, rho_dev, grad_dev, 1, (cudaStream_t)stream);
  }
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_density_grad");
}

srn_status srn_input_backward(srn_ctx* ctx, const float* pts_dev, int n, float time, const float* dout_dev,
                              float* dpts_dev, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || (n > 0 && (!pts_dev || !dout_dev || !dpts_dev)))
    return fail(SRN_ERR_INVALID_ARG, "points, dout and dpts are required");
  srn_status st = use_device(ctx);
  if (st) return st;
  cudaError_t e = launch_eval_fp32(make_net(ctx), pts_dev, n, time, nullptr, dpts_dev, 2, (cudaStream_t)stream,
                                   dout_dev);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_input_backward");
}

srn_status srn_backward(srn_ctx* ctx, const float* pts_dev, int n, float time, const float* dout_dev,
                        float* dgrid_dev, float* dweights_dev, float* dbiases_dev, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || n > ctx->cfg.max_fit_points)
    return fail(SRN_ERR_INVALID_ARG, "n must be in [0, max_fit_points=%d]", ctx->cfg.max_fit_points);
  if (ctx->cfg.max_fit_points < 1) return fail(SRN_ERR_INVALID_ARG, "context was created without fit scratch");
  if (n > 0 && (!pts_dev || !dout_dev)) return fail(SRN_ERR_INVALID_ARG, "points and dout are required");
  if (!fit_supported(make_net(ctx))) return fail(SRN_ERR_UNSUPPORTED, "backward does not implement this shape");
  if (!dgrid_dev || !dweights_dev || !dbiases_dev) return fail(SRN_ERR_INVALID_ARG, "gradient outputs are required");
  srn_status st = use_device(ctx);
  if (st) return st;
  cudaError_t e = launch_backward(ctx->fit, make_net(ctx), pts_dev, n, time, dout_dev, dgrid_dev, dweights_dev,
                                  dbiases_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_backward");
}

}  // extern "C"

namespace {

// Validation and argument set shared by srn_fit_step and srn_fit_steps.
srn_status make_fit_args(srn_ctx* ctx, const float* volume_dev, const int dims[3], int n_points, uint64_t seed,
                         int step, float time, float lr_grid, float lr_net, float grad_weight, float grad_scale,
                         float* loss_dev, FitArgs* out) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (!volume_dev || !dims || dims[0] < 2 || dims[1] < 2 || dims[2] < 2)
    return fail(SRN_ERR_INVALID_ARG, "volume with dims >= 2 is required");
  if (n_points < 1 || n_points > ctx->cfg.max_fit_points)
    return fail(SRN_ERR_INVALID_ARG, "n_points must be in [1, max_fit_points=%d]", ctx->cfg.max_fit_points);
  if (step < 0) return fail(SRN_ERR_INVALID_ARG, "step must be >= 0");
  if (!ctx->prm.adam_m || !ctx->prm.adam_v) return fail(SRN_ERR_INVALID_ARG, "Adam moments are required");
  if (!loss_dev) return fail(SRN_ERR_INVALID_ARG, "loss_dev is required");
  if (!fit_supported(make_net(ctx))) return fail(SRN_ERR_UNSUPPORTED, "fit does not implement this shape");
  if (ctx->cfg.out_dim == 4 && !(grad_scale == grad_scale && grad_weight >= 0.0f))
    return fail(SRN_ERR_INVALID_ARG, "grad_weight must be >= 0");
  if (!(lr_grid >= 0.0f) || !(lr_net >= 0.0f)) return fail(SRN_ERR_INVALID_ARG, "learning rates must be >= 0");
  if (ctx->cdf_active && !adaptive_fits(n_points, ctx->cdf_res))
    return fail(SRN_ERR_UNSUPPORTED, "n_points too large for 64-bit adaptive sampling at this resolution");
  FitArgs a{};
  a.vol = VolDev{volume_dev, dims[0], dims[1], dims[2]};
  a.n = n_points;
  a.seed = seed;
  a.step = step;
  a.time = time;
  a.lr_grid = lr_grid;
  a.lr_net = lr_net;
  a.grad_weight = grad_weight;
  a.grad_scale = grad_scale;
  a.loss = loss_dev;
  a.status = ctx->status;
  a.grid_h = reinterpret_cast<__half*>(ctx->prm.grid_h);
  a.weights_h = reinterpret_cast<__half*>(ctx->prm.weights_h);
  a.grid_exp = reinterpret_cast<const int*>(ctx->status + 4);
  a.adam_m = ctx->prm.adam_m;
  a.adam_v = ctx->prm.adam_v;
  a.grid = ctx->prm.grid;
  a.weights = ctx->prm.weights;
  a.biases = ctx->prm.biases;
  a.cdf = ctx->cdf_active ? ctx->cdf : nullptr;
  a.cdf_res = ctx->cdf_res;
  a.step_ptr = nullptr;
  a.stall_test = test_stall();
  *out = a;
  return SRN_OK;
}

// One fit step (Section 5.2 loss, Adam update) plus the 8-bit grid refresh.
cudaError_t enqueue_fit_step(srn_ctx* ctx, const FitArgs& a, cudaStream_t st) {
  const NetDev net = make_net(ctx);
  cudaError_t e = launch_fit_step(ctx->fit, net, a, st);
  if (e == cudaSuccess && ctx->cfg.grid_u8)
    e = launch_quantize_grid(net.grid, net_grid_count(net) / net.F, net.F, (uint8_t*)ctx->prm.grid_q,
                             ctx->prm.grid_qp, st);
  return e;
}

// Every field the graph bakes in, the step excepted (it is read from device memory).
bool same_graph_args(const FitArgs& x, const FitArgs& y) {
  return x.vol.vol == y.vol.vol && x.vol.nx == y.vol.nx && x.vol.ny == y.vol.ny && x.vol.nz == y.vol.nz &&
         x.n == y.n && x.seed == y.seed && memcmp(&x.time, &y.time, sizeof(float)) == 0 &&
         memcmp(&x.lr_grid, &y.lr_grid, sizeof(float)) == 0 && memcmp(&x.lr_net, &y.lr_net, sizeof(float)) == 0 &&
         memcmp(&x.grad_weight, &y.grad_weight, sizeof(float)) == 0 &&
         memcmp(&x.grad_scale, &y.grad_scale, sizeof(float)) == 0 && x.loss == y.loss && x.grid_h == y.grid_h &&
         x.weights_h == y.weights_h && x.adam_m == y.adam_m && x.adam_v == y.adam_v && x.grid == y.grid &&
         x.weights == y.weights && x.biases == y.biases && x.cdf == y.cdf && x.cdf_res == y.cdf_res && x.stall_test == y.stall_test;
}

// Captures one step (fit step, whose Adam kernel advances the step index,
// and the 8-bit grid refresh) on the context's own stream into
// ctx->graph_exec.
cudaError_t capture_fit_graph(srn_ctx* ctx, const FitArgs& a) {
  if (ctx->graph_exec) {
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
  }
  cudaError_t e = cudaSuccess;
  if (!ctx->graph_stream) e = cudaStreamCreateWithFlags(&ctx->graph_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  // relaxed: the launchers set kernel attributes (shared-memory size) while capturing
  e = cudaStreamBeginCapture(ctx->graph_stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  const cudaError_t le = enqueue_fit_step(ctx, a, ctx->graph_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(ctx->graph_stream, &g);  // always ends the capture
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e == cudaSuccess) ctx->graph_key = a;
  else ctx->graph_exec = nullptr;
  return e;
}

}  // namespace

extern "C" {

srn_status srn_fit_step(srn_ctx* ctx, const float* volume_dev, const int dims[3], int n_points, uint64_t seed,
                        int step, float time, float lr_grid, float lr_net, float grad_weight, float grad_scale,
                        float* loss_dev, void* stream) {
  FitArgs a;
  srn_status st = make_fit_args(ctx, volume_dev, dims, n_points, seed, step, time, lr_grid, lr_net, grad_weight,
                                grad_scale, loss_dev, &a);
  if (st) return st;
  st = use_device(ctx);
  if (st) return st;
  cudaError_t e = enqueue_fit_step(ctx, a, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_fit_step");
}

srn_status srn_fit_steps(srn_ctx* ctx, const float* volume_dev, const int dims[3], int n_points, uint64_t seed,
                         int first_step, int n_steps, float time, float lr_grid, float lr_net, float grad_weight,
                         float grad_scale, float* loss_dev, void* stream) {
  FitArgs a;
  srn_status st = make_fit_args(ctx, volume_dev, dims, n_points, seed, first_step, time, lr_grid, lr_net,
                                grad_weight, grad_scale, loss_dev, &a);
  if (st) return st;
  if (n_steps < 0 || first_step > INT_MAX - n_steps)
    return fail(SRN_ERR_INVALID_ARG, "n_steps must be >= 0 and first_step + n_steps must fit an int");
  if (n_steps == 0) return SRN_OK;
  st = use_device(ctx);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int* step_dev = reinterpret_cast<int*>(ctx->status + 1);
  a.step_ptr = step_dev;
  cudaError_t e = cudaSuccess;
  // capturing records the launches without running them: nothing executes
  // before the replays below, which are ordered on `stream`
  if (!ctx->graph_exec || !same_graph_args(a, ctx->graph_key)) e = capture_fit_graph(ctx, a);
  if (e == cudaSuccess) e = launch_step_counter(step_dev, first_step, ctx->fit.flag, s);
  for (int i = 0; i < n_steps && e == cudaSuccess; ++i) e = cudaGraphLaunch(ctx->graph_exec, s);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_fit_steps");
}

srn_status srn_sync_status(srn_ctx* ctx, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  unsigned int word = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&word, ctx->status, sizeof(word), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "srn_sync_status");
  if (word == SRN_ERR_NONFINITE)
    return fail(SRN_ERR_NONFINITE, "a fit step produced a non-finite loss or gradient, or the FP16 path a non-finite output");
  if (word == SRN_ERR_TIMEOUT) return fail(SRN_ERR_TIMEOUT, "a bounded device wait gave up");
  if (word != 0) return fail(SRN_ERR_INTERNAL, "device status word %u", word);
  return SRN_OK;
}

srn_status srn_image_mse(const float* a_dev, const float* b_dev, long long n_pixels, double* mse_dev,
                         void* stream) {
  if (n_pixels < 0 || !mse_dev || (n_pixels > 0 && (!a_dev || !b_dev)))
    return fail(SRN_ERR_INVALID_ARG, "bad image arguments");
  if (!aligned16(a_dev) || !aligned16(b_dev)) return fail(SRN_ERR_INVALID_ARG, "images must be 16-byte aligned");
  cudaError_t e = launch_image_mse(a_dev, b_dev, n_pixels, mse_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_image_mse");
}

srn_status srn_image_ssim(const float* a_dev, const float* b_dev, int width, int height, double* ssim_dev,
                          void* stream) {
  if (width < 1 || height < 1 || !a_dev || !b_dev || !ssim_dev)
    return fail(SRN_ERR_INVALID_ARG, "images of at least 1 x 1 pixels and the output are required");
  if (!aligned16(a_dev) || !aligned16(b_dev)) return fail(SRN_ERR_INVALID_ARG, "images must be 16-byte aligned");
  cudaError_t e = launch_image_ssim(a_dev, b_dev, width, height, ssim_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_image_ssim");
}

namespace {

const char kCkptMagic[8] = {'S', 'R', 'N', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 2;

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t shape[10];  // grid_res, feat, n_fourier, layers, width, out_dim, activation, n_keyframes, time_input,
                      // has_adam
  int32_t step;
  uint64_t n_grid, n_weights, n_biases;
};

void ckpt_shape(const srn_ctx* ctx, int32_t shape[10]) {
  const srn_config& c = ctx->cfg;
  shape[0] = c.grid_res; shape[1] = c.feat; shape[2] = c.n_fourier; shape[3] = c.layers; shape[4] = c.width;
  shape[5] = c.out_dim; shape[6] = c.activation; shape[7] = c.n_keyframes; shape[8] = c.time_input;
  shape[9] = (ctx->prm.adam_m && ctx->prm.adam_v) ? 1 : 0;
}

}  // namespace

srn_status srn_save(srn_ctx* ctx, const char* path, int step) {
  if (!ctx || !path) return fail(SRN_ERR_INVALID_ARG, "ctx and path are required");
  srn_status st = use_device(ctx);
  if (st) return st;
  const NetDev n = make_net(ctx);
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.version = kCkptVersion;
  ckpt_shape(ctx, h.shape);
  h.step = step;
  h.n_grid = net_grid_count(n);
  h.n_weights = net_weight_count(n);
  h.n_biases = net_bias_count(n);
  const size_t total = h.n_grid + h.n_weights + h.n_biases;
  float* host = (float*)malloc(sizeof(float) * total * (h.shape[9] ? 3 : 1));
  if (!host) return fail(SRN_ERR_INTERNAL, "out of host memory");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host, ctx->prm.grid, sizeof(float) * h.n_grid, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(host + h.n_grid, ctx->prm.weights, sizeof(float) * h.n_weights, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(host + h.n_grid + h.n_weights, ctx->prm.biases, sizeof(float) * h.n_biases,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h.shape[9]) {
    e = cudaMemcpy(host + total, ctx->prm.adam_m, sizeof(float) * total, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(host + 2 * total, ctx->prm.adam_v, sizeof(float) * total, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) {
    free(host);
    return cuda_fail(e, "srn_save");
  }
  FILE* f = fopen(path, "wb");
  if (!f) {
    free(host);
    return fail(SRN_ERR_INVALID_ARG, "cannot open %s for writing", path);
  }
  const size_t nfl = total * (h.shape[9] ? 3 : 1);
  const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(host, sizeof(float), nfl, f) == nfl;
  free(host);
  if (fclose(f) != 0 || !ok) return fail(SRN_ERR_INTERNAL, "short write to %s", path);
  return SRN_OK;
}

srn_status srn_load(srn_ctx* ctx, const char* path, int* step_out) {
  if (!ctx || !path) return fail(SRN_ERR_INVALID_ARG, "ctx and path are required");
  srn_status st = use_device(ctx);
  if (st) return st;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(SRN_ERR_INVALID_ARG, "cannot open %s", path);
  CkptHeader h;
  if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion) {
    fclose(f);
    return fail(SRN_ERR_INVALID_ARG, "%s is not an srn checkpoint of version %u", path, kCkptVersion);
  }
  int32_t shape[10];
  ckpt_shape(ctx, shape);
  const NetDev n = make_net(ctx);
  if (memcmp(shape, h.shape, sizeof(int32_t) * 9) != 0 || h.n_grid != net_grid_count(n) ||
      h.n_weights != net_weight_count(n) || h.n_biases != net_bias_count(n)) {
    fclose(f);
    return fail(SRN_ERR_INVALID_ARG, "checkpoint %s has a different network shape", path);
  }
  const size_t total = h.n_grid + h.n_weights + h.n_biases;
  const size_t nfl = total * (h.shape[9] ? 3 : 1);
  float* host = (float*)malloc(sizeof(float) * nfl);
  if (!host) {
    fclose(f);
    return fail(SRN_ERR_INTERNAL, "out of host memory");
  }
  const bool ok = fread(host, sizeof(float), nfl, f) == nfl;
  fclose(f);
  if (!ok) {
    free(host);
    return fail(SRN_ERR_INVALID_ARG, "checkpoint %s is truncated", path);
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(ctx->prm.grid, host, sizeof(float) * h.n_grid, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->prm.weights, host + h.n_grid, sizeof(float) * h.n_weights, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->prm.biases, host + h.n_grid + h.n_weights, sizeof(float) * h.n_biases,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && h.shape[9] && shape[9]) {
    e = cudaMemcpy(ctx->prm.adam_m, host + total, sizeof(float) * total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->prm.adam_v, host + 2 * total, sizeof(float) * total, cudaMemcpyHostToDevice);
  }
  free(host);
  if (e != cudaSuccess) return cuda_fail(e, "srn_load");
  if (ctx->prm.grid_h && ctx->prm.weights_h) {
    e = write_half_copies(ctx, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "srn_load");
  }
  if (step_out) *step_out = h.step;
  return SRN_OK;
}

srn_status srn_error_grid(srn_ctx* ctx, const float* volume_dev, const int dims[3], int res, int samples_per_voxel,
                          uint64_t seed, float time, float* err_dev, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (!volume_dev || !dims || dims[0] < 2 || dims[1] < 2 || dims[2] < 2)
    return fail(SRN_ERR_INVALID_ARG, "volume with dims >= 2 is required");
  if (res < 2 || res > 256) return fail(SRN_ERR_INVALID_ARG, "res must be in [2, 256]");
  if (samples_per_voxel < 1 || samples_per_voxel > 64)
    return fail(SRN_ERR_INVALID_ARG, "samples_per_voxel must be in [1, 64]");
  if (!err_dev) return fail(SRN_ERR_INVALID_ARG, "err_dev is required");
  srn_status st = use_device(ctx);
  if (st) return st;
  cudaError_t e = launch_error_grid(make_net(ctx), VolDev{volume_dev, dims[0], dims[1], dims[2]}, res,
                                    samples_per_voxel, seed, time, err_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_error_grid");
}

srn_status srn_fit_set_sampling(srn_ctx* ctx, const float* err_dev, int res, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (!err_dev) {
    ctx->cdf_active = false;
    return SRN_OK;
  }
  if (res < 2 || res > 256) return fail(SRN_ERR_INVALID_ARG, "res must be in [2, 256]");
  srn_status st = use_device(ctx);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = (long long)res * res * res;
  const long long nb = (n + kCdfBlock - 1) / kCdfBlock;
  cudaError_t e = cudaSuccess;
  if (!ctx->cdf_flags) e = cudaMalloc((void**)&ctx->cdf_flags, 2 * sizeof(unsigned int));
  if (e == cudaSuccess) e = launch_error_max(err_dev, n, ctx->cdf_flags, s);
  unsigned int flags[2] = {0u, 0u};
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags, ctx->cdf_flags, sizeof(flags), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "srn_fit_set_sampling");
  if (flags[0]) return fail(SRN_ERR_INVALID_ARG, "error grid has a negative or non-finite entry");
  if (flags[1] == 0u) {
    ctx->cdf_active = false;  // all zero: uniform sampling
    return SRN_OK;
  }
  if ((size_t)(n + 1) > ctx->cdf_cap) {
    if (ctx->cdf) cudaFree(ctx->cdf);
    if (ctx->cdf_bsum) cudaFree(ctx->cdf_bsum);
    ctx->cdf = nullptr;
    ctx->cdf_bsum = nullptr;
    ctx->cdf_cap = 0;
    ctx->cdf_active = false;
    e = cudaMalloc((void**)&ctx->cdf, sizeof(unsigned long long) * (size_t)(n + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->cdf_bsum, sizeof(unsigned long long) * (size_t)nb);
    if (e != cudaSuccess) return cuda_fail(e, "srn_fit_set_sampling");
    ctx->cdf_cap = (size_t)(n + 1);
  }
  e = launch_build_cdf(err_dev, n, ctx->cdf_flags, ctx->cdf, ctx->cdf_bsum, s);
  if (e != cudaSuccess) return cuda_fail(e, "srn_fit_set_sampling");
  ctx->cdf_res = res;
  ctx->cdf_active = true;
  return SRN_OK;
}

srn_status srn_fit_points(srn_ctx* ctx, int n_points, uint64_t seed, int step, float* pts_dev, void* stream) {
  if (!ctx) return fail(SRN_ERR_INVALID_ARG, "ctx is NULL");
  if (n_points < 0 || (n_points > 0 && !pts_dev)) return fail(SRN_ERR_INVALID_ARG, "bad n_points / pts_dev");
  if (step < 0) return fail(SRN_ERR_INVALID_ARG, "step must be >= 0");
  if (ctx->cdf_active && !adaptive_fits(n_points, ctx->cdf_res))
    return fail(SRN_ERR_UNSUPPORTED, "n_points too large for 64-bit adaptive sampling at this resolution");
  srn_status st = use_device(ctx);
  if (st) return st;
  cudaError_t e = launch_fit_points(ctx->cdf_active ? ctx->cdf : nullptr, ctx->cdf_res, seed, step, n_points,
                                    pts_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_fit_points");
}

srn_status srn_density_mse(const float* a_dev, const float* b_dev, long long n, double* mse_dev, void* stream) {
  if (n < 0 || !mse_dev || (n > 0 && (!a_dev || !b_dev))) return fail(SRN_ERR_INVALID_ARG, "bad arrays");
  cudaError_t e = launch_density_mse(a_dev, b_dev, n, mse_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_density_mse");
}

srn_status srn_resample(const float* src_dev, const int src_dims[3], float* dst_dev, const int dst_dims[3],
                        void* stream) {
  if (!src_dev || !dst_dev || !src_dims || !dst_dims) return fail(SRN_ERR_INVALID_ARG, "arrays and dims required");
  for (int a = 0; a < 3; ++a)
    if (src_dims[a] < 2 || dst_dims[a] < 1) return fail(SRN_ERR_INVALID_ARG, "source dims >= 2, target dims >= 1");
  cudaError_t e = launch_resample(src_dev, src_dims, dst_dev, dst_dims, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_resample");
}

srn_status srn_lowpass_resample(const float* volume_dev, const int dims[3], int M, float* tmp_dev, float* out_dev,
                                void* stream) {
  if (!volume_dev || !dims || !tmp_dev || !out_dev) return fail(SRN_ERR_INVALID_ARG, "arrays and dims required");
  if (dims[0] < 2 || dims[1] < 2 || dims[2] < 2 || M < 2) return fail(SRN_ERR_INVALID_ARG, "dims and M must be >= 2");
  if (!lowpass_supported(dims, M)) return fail(SRN_ERR_UNSUPPORTED, "filter wider than 257 taps");
  cudaError_t e = launch_lowpass_resample(volume_dev, dims, M, tmp_dev, out_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_lowpass_resample");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// srn_backward_static: the backward without any allocation, for callers that
// cannot call cudaMalloc (device memory owned by another allocator, frame
// loops that must not take an allocation's synchronization).  Its scratch is
// the file-scope device array below.  In host code the array's name is only
// a host-side stand-in for the symbol, never a device address: the address is
// looked up with cudaGetSymbolAddress once per device (with that device
// current) and passed to the kernels.

namespace {

__device__ __align__(256) unsigned char g_static_scratch[SRN_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

srn_status static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(SRN_ERR_UNSUPPORTED, "device index %d is out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return SRN_OK;
}

// Carves the fit scratch of n points out of the static area; returns the
// bytes needed (which may exceed the area).
size_t carve_static(FitScratch& s, const NetDev& net, int n, unsigned char* base, int sms) {
  memset(&s, 0, sizeof(s));
  s.max_points = n;
  s.n_cells = (size_t)(net.R - 1) * (net.R - 1) * (net.R - 1);
  s.n_entries = net_weight_count(net) + net_bias_count(net);
  s.n_grid = net_grid_count(net);
  s.max_cta = std::max(1, std::min(sms, (n + 127) / 128));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    void* p = (void*)((uintptr_t)base + off);
    off = (off + bytes + 255) & ~(size_t)255;
    return p;
  };
  const size_t nn = (size_t)std::max(n, 1);
  s.pts = (float*)take(sizeof(float) * 3 * nn);
  s.dz = (float*)take(sizeof(float) * net.F * nn);
  s.key = (unsigned int*)take(sizeof(unsigned int) * nn);
  s.key_alt = (unsigned int*)take(sizeof(unsigned int) * nn);
  s.idx = (unsigned int*)take(sizeof(unsigned int) * nn);
  s.idx_alt = (unsigned int*)take(sizeof(unsigned int) * nn);
  s.radix_bins = 256;  // two 8-bit passes: the smaller histogram keeps the static area's batch
  const size_t hist_n = 256 * ((nn + 2047) / 2048);
  s.hist = (unsigned int*)take(sizeof(unsigned int) * (hist_n + hist_n / 8192 + 1));
  s.digit_totals = (unsigned int*)take(sizeof(unsigned int) * 256);
  s.cell_start = (unsigned int*)take(sizeof(unsigned int) * (s.n_cells + 1));
  s.part = (float*)take(sizeof(float) * (size_t)s.max_cta * (s.n_entries + 1));
  s.flag = (unsigned int*)take(sizeof(unsigned int) * 4);
  s.grads = nullptr;  // the backward writes straight into the caller's outputs
  return off;
}

}  // namespace

extern "C" srn_status srn_backward_static(const srn_config* cfg, const srn_params* params, const float* pts_dev,
                                          int n, float time, const float* dout_dev, float* dgrid_dev,
                                          float* dweights_dev, float* dbiases_dev, void* stream) {
  srn_status st = check_config(cfg);
  if (st) return st;
  st = check_params(cfg, params);
  if (st) return st;
  if (n < 0) return fail(SRN_ERR_INVALID_ARG, "n must be >= 0");
  if (n > 0 && (!pts_dev || !dout_dev)) return fail(SRN_ERR_INVALID_ARG, "points and dout are required");
  if (!dgrid_dev || !dweights_dev || !dbiases_dev) return fail(SRN_ERR_INVALID_ARG, "gradient outputs are required");
  srn_ctx view;  // a stack description of the network; nothing is allocated
  memset(&view, 0, sizeof(view));
  view.cfg = *cfg;
  view.prm = *params;
  const NetDev net = make_net(&view);
  if (!fit_supported(net)) return fail(SRN_ERR_UNSUPPORTED, "backward does not implement this shape");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "srn_backward_static");
  FitScratch s;
  const size_t need = carve_static(s, net, n, nullptr, sms);
  if (need > (size_t)SRN_STATIC_SCRATCH_BYTES) {
    // largest n that fits this network shape
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = lo + (hi - lo + 1) / 2;
      FitScratch t;
      if (carve_static(t, net, mid, nullptr, sms) <= (size_t)SRN_STATIC_SCRATCH_BYTES) lo = mid;
      else hi = mid - 1;
    }
    return fail(SRN_ERR_INVALID_ARG, "n = %d needs %zu bytes of scratch; the static area holds %u bytes "
                "(at most n = %d for this network)", n, need, (unsigned)SRN_STATIC_SCRATCH_BYTES, lo);
  }
  void* base = nullptr;
  st = static_scratch_address(&base);
  if (st) return st;
  carve_static(s, net, n, (unsigned char*)base, sms);
  e = launch_backward(s, net, pts_dev, n, time, dout_dev, dgrid_dev, dweights_dev, dbiases_dev,
                      (cudaStream_t)stream);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "srn_backward_static");
}
