/*
 * FP64 CPU oracle for the fV-SRN render / fit path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the GPU path computes, used to check it.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the product library never links, loads or calls it, and it shares no
 * code, header or table with the CUDA sources.
 *
 * Paper: Weiss, Hermüller, Westermann, "Fast Neural Representations for Direct
 * Volume Rendering" (fV-SRN), arXiv 2112.01579.  Citations below name the
 * paper's section / equation.  Where the paper is silent the reading taken is
 * stated at the function ("Reading: ...").
 *
 * Everything is double precision.  Parameters given to the oracle are the
 * exact values the GPU uses (FP16 copies widened exactly), so differences
 * between the two are rounding of the GPU arithmetic only.
 *
 * Parity status per function (what pins it; the pins live in the test suite):
 *   orc_philox4x32_10      Random123 known-answer vectors
 *   orc_trilinear(_grad)   affine fields reproduced exactly; corner values
 *   orc_net_forward        selector-weight closed forms, zero last layer,
 *                          Fourier rows vs sin/cos of Eq. 1, Eq. 3 SnakeAlt
 *   orc_net_backward       brute-force central finite differences (FP64)
 *   orc_net_input_grad     brute-force central finite differences (FP64)
 *   orc_render             constant slab exp(-kappa L); early-termination
 *                          step index; shaded linear ramp closed form
 *   orc_dvr_dense          Gaussian blob line integral via erf
 *   orc_fit_step           finite differences of the loss + torch.optim.Adam
 *   orc_error_grid         constant network vs constant / linear volume
 *                          closed forms; every sample inside its voxel
 *   orc_adaptive_cdf /     one-hot, uniform and 1:3 error grids give
 *   orc_adaptive_point     exactly proportional point counts (+-1); points
 *                          inside the chosen voxel; zero-error voxels empty
 *   orc_lowpass_resample   constant and affine fields preserved
 *   orc_psnr / orc_ssim    SSIM of constant images in closed form; identity
 * Head-mode training quality (loss design in the paper's missing supplement)
 * is parity unpinned beyond the pieces above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXW 256 /* widest layer input / output the oracle supports */
#define ORC_MAXL 16  /* deepest network */

enum { ORC_ACT_SINE = 0, ORC_ACT_SNAKEALT = 1 };
enum { ORC_SHADE_NONE = 0, ORC_SHADE_ADJOINT = 1, ORC_SHADE_FD = 2, ORC_SHADE_HEAD = 3 };

/* Network description (Section 3 layer equation, Section 4.2 latent grid,
 * Section 7 keyframes).  Layer i maps d_i -> d_{i+1} with
 * d_0 = 3 + 2m + F, d_1..d_{l-1} = c, d_l = D.  W_i is row-major
 * [d_{i+1}][d_i]; layers and biases are packed back to back.
 * grid is [nkey][R][R][R][F] with x fastest and channels innermost. */
typedef struct {
  int R, F, m, l, c, D, act, nkey;
  int time_input;          /* 1: the time value is one more input after z (Section 7 "direct") */
  const double* key_times; /* nkey increasing keyframe times (nkey > 1) */
  double* grid;
  const double* fourier; /* m x 3 */
  double* W;
  double* b;
} orc_net;

typedef struct {
  double eye[3], target[3], up[3];
  double fovy; /* vertical field of view, radians */
} orc_camera;

typedef struct {
  int n;
  const double* pos;  /* n sorted control points in [0,1] */
  const double* rgba; /* n x 4 */
  double opacity_scale;
} orc_tf;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC 2011): ten rounds of the Philox S-box with the
 * published multipliers and Weyl key increments. */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c0, &hi0, &lo0);
    mulhilo32(M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Training-point sampler of the fit (Section 5 world-space training; the
 * paper draws uniform random positions).  Reading: point j of step s uses
 * counter (j, s, 0x5352, 0) and key (seed_lo, seed_hi); coordinate a is
 * (word_a >> 8) * 2^-24, a multiple of 2^-24 in [0,1) that FP32 holds exactly. */
void orc_sample_point(uint64_t seed, int step, int j, double p[3]) {
  uint32_t ctr[4] = {(uint32_t)j, (uint32_t)step, 0x5352u, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  for (int a = 0; a < 3; ++a) p[a] = (double)(o[a] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* Reading of Section 4.2 ("R vertices along each axis", values interpolated
 * trilinearly inside each cell): vertex-aligned, g = p (n-1), the cell index
 * is floor(g) limited to [0, n-2], so p = 1 lies in the last cell. */
static void cell_coord(double p, int n, int* i0, double* f) {
  double g = p * (double)(n - 1);
  int i = (int)floor(g);
  if (i > n - 2) i = n - 2;
  if (i < 0) i = 0;
  *i0 = i;
  *f = g - (double)i;
}

/* Trilinear interpolation of a C-channel field stored [z][y][x][C]. */
void orc_trilinear(const double* vol, int nx, int ny, int nz, int C, const double p_in[3], double* out) {
  double p[3] = {clamp01(p_in[0]), clamp01(p_in[1]), clamp01(p_in[2])};
  int ix, iy, iz;
  double fx, fy, fz;
  cell_coord(p[0], nx, &ix, &fx);
  cell_coord(p[1], ny, &iy, &fy);
  cell_coord(p[2], nz, &iz, &fz);
  for (int ch = 0; ch < C; ++ch) out[ch] = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
        size_t v = (((size_t)(iz + dz) * ny + (iy + dy)) * nx + (ix + dx)) * (size_t)C;
        for (int ch = 0; ch < C; ++ch) out[ch] += w * vol[v + ch];
      }
}

/* Gradient of the trilinear interpolant with respect to p (one-sided at cell
 * faces, following the cell choice of cell_coord).  grad is C x 3. */
void orc_trilinear_grad(const double* vol, int nx, int ny, int nz, int C, const double p_in[3], double* grad) {
  double p[3] = {clamp01(p_in[0]), clamp01(p_in[1]), clamp01(p_in[2])};
  int ix, iy, iz;
  double fx, fy, fz;
  cell_coord(p[0], nx, &ix, &fx);
  cell_coord(p[1], ny, &iy, &fy);
  cell_coord(p[2], nz, &iz, &fz);
  for (int k = 0; k < 3 * C; ++k) grad[k] = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double wx = dx ? fx : 1.0 - fx, wy = dy ? fy : 1.0 - fy, wz = dz ? fz : 1.0 - fz;
        double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0, sz = dz ? 1.0 : -1.0;
        double gx = sx * wy * wz * (double)(nx - 1);
        double gy = wx * sy * wz * (double)(ny - 1);
        double gz = wx * wy * sz * (double)(nz - 1);
        size_t v = (((size_t)(iz + dz) * ny + (iy + dy)) * nx + (ix + dx)) * (size_t)C;
        for (int ch = 0; ch < C; ++ch) {
          grad[3 * ch + 0] += gx * vol[v + ch];
          grad[3 * ch + 1] += gy * vol[v + ch];
          grad[3 * ch + 2] += gz * vol[v + ch];
        }
      }
}

/* ------------------------------------------------------------------------ */
static int layer_in(const orc_net* n, int i) { return i == 0 ? 3 + 2 * n->m + n->F + n->time_input : n->c; }
static int layer_out(const orc_net* n, int i) { return i == n->l - 1 ? n->D : n->c; }

/* Section 7: keyframe latent grids, linearly interpolated in time between the
 * two bracketing keyframes.  Reading: times outside the keyframe range clamp
 * to the first / last keyframe. */
static void time_weights(const orc_net* n, double t, int* k0, double* f) {
  if (n->nkey <= 1) { *k0 = 0; *f = 0.0; return; }
  const double* kt = n->key_times;
  if (t <= kt[0]) { *k0 = 0; *f = 0.0; return; }
  if (t >= kt[n->nkey - 1]) { *k0 = n->nkey - 2; *f = 1.0; return; }
  int k = 0;
  while (k < n->nkey - 2 && t >= kt[k + 1]) ++k;
  *k0 = k;
  *f = (t - kt[k]) / (kt[k + 1] - kt[k]);
}

static void latent(const orc_net* n, const double p[3], double t, double* z) {
  size_t gsz = (size_t)n->R * n->R * n->R * n->F;
  int k0;
  double f;
  time_weights(n, t, &k0, &f);
  orc_trilinear(n->grid + (size_t)k0 * gsz, n->R, n->R, n->R, n->F, p, z);
  if (n->nkey > 1) {
    double z1[ORC_MAXW];
    orc_trilinear(n->grid + (size_t)(k0 + 1) * gsz, n->R, n->R, n->R, n->F, p, z1);
    for (int ch = 0; ch < n->F; ++ch) z[ch] = (1.0 - f) * z[ch] + f * z1[ch];
  }
}

/* Eq. 3 (SnakeAlt) and the sine activation; derivatives for the backward. */
static double act_f(int act, double x) {
  if (act == ORC_ACT_SNAKEALT) { double s = sin(x); return 0.5 * x + s * s; }
  return sin(x);
}
static double act_df(int act, double x) {
  if (act == ORC_ACT_SNAKEALT) return 0.5 + 2.0 * sin(x) * cos(x);
  return cos(x);
}

typedef struct {
  double v[ORC_MAXL + 1][ORC_MAXW]; /* v[0] = input vector, v[i+1] = layer i output */
  double h[ORC_MAXL][ORC_MAXW];     /* pre-activations */
  double e[ORC_MAXW];               /* Fourier arguments F p */
  double p[3];                      /* clamped position */
} orc_trace;

/* Forward pass (Section 3 layer equation; Eq. 1-2 Fourier features; Section
 * 4.2 latent vector as additional input).  Reading: input order
 * v0 = [p, sin(F p), cos(F p), z]; activation after every layer but the
 * last; the last layer is linear. */
static void forward(const orc_net* n, const double p_in[3], double t, orc_trace* tr) {
  for (int a = 0; a < 3; ++a) tr->p[a] = clamp01(p_in[a]);
  double* v0 = tr->v[0];
  v0[0] = tr->p[0]; v0[1] = tr->p[1]; v0[2] = tr->p[2];
  for (int k = 0; k < n->m; ++k) {
    const double* Fk = n->fourier + 3 * k;
    double e = Fk[0] * tr->p[0] + Fk[1] * tr->p[1] + Fk[2] * tr->p[2];
    tr->e[k] = e;
    v0[3 + k] = sin(e);
    v0[3 + n->m + k] = cos(e);
  }
  latent(n, tr->p, t, v0 + 3 + 2 * n->m);
  /* Section 7 "direct" time encoding: the time is an additional scalar input.
   * Reading: the time value exactly as given to the call. */
  if (n->time_input) v0[3 + 2 * n->m + n->F] = t;
  const double* W = n->W;
  const double* b = n->b;
  for (int i = 0; i < n->l; ++i) {
    int din = layer_in(n, i), dout = layer_out(n, i);
    for (int o = 0; o < dout; ++o) {
      double h = b[o];
      for (int j = 0; j < din; ++j) h += W[(size_t)o * din + j] * tr->v[i][j];
      tr->h[i][o] = h;
      tr->v[i + 1][o] = (i < n->l - 1) ? act_f(n->act, h) : h;
    }
    W += (size_t)dout * din;
    b += dout;
  }
}

int orc_net_check(const orc_net* n) {
  if (n->l < 1 || n->l > ORC_MAXL) return 1;
  if (3 + 2 * n->m + n->F + 1 > ORC_MAXW || n->c > ORC_MAXW || n->D > ORC_MAXW) return 1;
  if (n->time_input != 0 && n->time_input != 1) return 1;
  if (n->R < 2 || n->nkey < 1 || n->D < 1) return 1;
  return 0;
}

/* Network output at n_pts positions (pts n x 3), time t; out is n x D. */
void orc_net_forward(const orc_net* n, const double* pts, int n_pts, double t, double* out) {
  #pragma omp parallel for schedule(dynamic, 64)
  for (int j = 0; j < n_pts; ++j) {
    orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
    forward(n, pts + 3 * j, t, tr);
    for (int d = 0; d < n->D; ++d) out[(size_t)j * n->D + d] = tr->v[n->l][d];
    free(tr);
  }
}

/* Backpropagation of an output adjoint dout (D values) through one traced
 * evaluation.  Accumulates into dW, db (packed like W, b) and dgrid (like
 * grid) when non-null; writes dv0 (gradient w.r.t. the input vector). */
static void backward(const orc_net* n, const orc_trace* tr, double t, const double* dout, double* dW, double* db,
                     double* dgrid, double* dv0) {
  double delta[ORC_MAXW], g[ORC_MAXW];
  size_t woff[ORC_MAXL + 1], boff[ORC_MAXL + 1];
  woff[0] = 0; boff[0] = 0;
  for (int i = 0; i < n->l; ++i) {
    woff[i + 1] = woff[i] + (size_t)layer_out(n, i) * layer_in(n, i);
    boff[i + 1] = boff[i] + (size_t)layer_out(n, i);
  }
  for (int o = 0; o < n->D; ++o) delta[o] = dout[o];
  for (int i = n->l - 1; i >= 0; --i) {
    int din = layer_in(n, i), dout_i = layer_out(n, i);
    const double* W = n->W + woff[i];
    for (int o = 0; o < dout_i; ++o) {
      if (dW) for (int j = 0; j < din; ++j) dW[woff[i] + (size_t)o * din + j] += delta[o] * tr->v[i][j];
      if (db) db[boff[i] + o] += delta[o];
    }
    for (int j = 0; j < din; ++j) {
      double s = 0.0;
      for (int o = 0; o < dout_i; ++o) s += W[(size_t)o * din + j] * delta[o];
      g[j] = s;
    }
    if (i > 0)
      for (int j = 0; j < din; ++j) delta[j] = g[j] * act_df(n->act, tr->h[i - 1][j]);
  }
  int d0 = layer_in(n, 0);
  if (dv0) for (int j = 0; j < d0; ++j) dv0[j] = g[j];
  if (dgrid) {
    /* the latent vector is a weighted sum of grid vertices (trilinear weights
     * times time weights), so its adjoint scatters back with the same weights */
    const double* dz = g + 3 + 2 * n->m;
    size_t gsz = (size_t)n->R * n->R * n->R * n->F;
    int k0;
    double f;
    time_weights(n, t, &k0, &f);
    int ix, iy, iz;
    double fx, fy, fz;
    cell_coord(tr->p[0], n->R, &ix, &fx);
    cell_coord(tr->p[1], n->R, &iy, &fy);
    cell_coord(tr->p[2], n->R, &iz, &fz);
    for (int kk = 0; kk < (n->nkey > 1 ? 2 : 1); ++kk) {
      double tw = (n->nkey > 1) ? (kk ? f : 1.0 - f) : 1.0;
      double* G = dgrid + (size_t)(k0 + kk) * gsz;
      for (int dz_ = 0; dz_ < 2; ++dz_)
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) {
            double w = tw * (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz_ ? fz : 1.0 - fz);
            size_t v = (((size_t)(iz + dz_) * n->R + (iy + dy)) * n->R + (ix + dx)) * (size_t)n->F;
            for (int ch = 0; ch < n->F; ++ch) G[v + ch] += w * dz[ch];
          }
    }
  }
}

/* Parameter gradients of sum_j <dout_j, net(p_j)>: dW, db, dgrid are
 * accumulated (caller zeroes them). */
void orc_net_backward(const orc_net* n, const double* pts, int n_pts, double t, const double* dout, double* dW,
                      double* db, double* dgrid) {
  orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
  for (int j = 0; j < n_pts; ++j) {
    forward(n, pts + 3 * j, t, tr);
    backward(n, tr, t, dout + (size_t)j * n->D, dW, db, dgrid, NULL);
  }
  free(tr);
}

/* Adjoint input gradient (Section 5 "Adjoint") of sum_d s_d out_d (s = dout;
 * NULL: s = e_0, i.e. d out_0 / d p) by backpropagation through the layers,
 * the Fourier features (d sin(e) = cos(e) F_k, d cos(e) = -sin(e) F_k) and
 * the trilinear latent grid. */
static void input_vjp_traced(const orc_net* n, const orc_trace* tr, double t, const double* seed, double grad[3]) {
  double dout[ORC_MAXW], dv0[ORC_MAXW];
  for (int d = 0; d < n->D; ++d) dout[d] = seed ? seed[d] : ((d == 0) ? 1.0 : 0.0);
  backward(n, tr, t, dout, NULL, NULL, NULL, dv0);
  for (int a = 0; a < 3; ++a) grad[a] = dv0[a];
  for (int k = 0; k < n->m; ++k) {
    double s = dv0[3 + k] * cos(tr->e[k]) - dv0[3 + n->m + k] * sin(tr->e[k]);
    for (int a = 0; a < 3; ++a) grad[a] += s * n->fourier[3 * k + a];
  }
  const double* dz = dv0 + 3 + 2 * n->m;
  size_t gsz = (size_t)n->R * n->R * n->R * n->F;
  int k0;
  double f;
  time_weights(n, t, &k0, &f);
  double* jac = (double*)malloc(sizeof(double) * 3 * n->F);
  for (int kk = 0; kk < (n->nkey > 1 ? 2 : 1); ++kk) {
    double tw = (n->nkey > 1) ? (kk ? f : 1.0 - f) : 1.0;
    orc_trilinear_grad(n->grid + (size_t)(k0 + kk) * gsz, n->R, n->R, n->R, n->F, tr->p, jac);
    for (int ch = 0; ch < n->F; ++ch)
      for (int a = 0; a < 3; ++a) grad[a] += tw * dz[ch] * jac[3 * ch + a];
  }
  free(jac);
}

static void input_grad_traced(const orc_net* n, const orc_trace* tr, double t, double grad[3]) {
  input_vjp_traced(n, tr, t, NULL, grad);
}

/* Density and its adjoint gradient at n_pts positions: rho n, grad n x 3. */
void orc_net_input_grad(const orc_net* n, const double* pts, int n_pts, double t, double* rho, double* grad) {
  #pragma omp parallel for schedule(dynamic, 64)
  for (int j = 0; j < n_pts; ++j) {
    orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
    forward(n, pts + 3 * j, t, tr);
    rho[j] = tr->v[n->l][0];
    input_grad_traced(n, tr, t, grad + 3 * (size_t)j);
    free(tr);
  }
}

/* Backward with respect to the positions: grad_j = sum_d dout_j[d]
 * d out_d / d p_j (n_pts x 3), dout n_pts x D. */
void orc_net_input_vjp(const orc_net* n, const double* pts, int n_pts, double t, const double* dout, double* grad) {
  #pragma omp parallel for schedule(dynamic, 64)
  for (int j = 0; j < n_pts; ++j) {
    orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
    forward(n, pts + 3 * j, t, tr);
    input_vjp_traced(n, tr, t, dout + (size_t)j * n->D, grad + 3 * (size_t)j);
    free(tr);
  }
}

/* ------------------------------------------------------------------------ */
/* Transfer function (Section 3: densities mapped to colour by a TF).
 * Reading: density clamped to [0,1]; piecewise-linear RGBA between sorted
 * control points, constant beyond the first / last point; the segment is the
 * one with pos[i] <= x < pos[i+1]; extinction kappa = A * opacity_scale. */
void orc_tf_eval(const orc_tf* tf, double rho, double rgba[4]) {
  double x = clamp01(rho);
  const double* P = tf->pos;
  const double* C = tf->rgba;
  int n = tf->n;
  if (x <= P[0]) { for (int k = 0; k < 4; ++k) rgba[k] = C[k]; return; }
  if (x >= P[n - 1]) { for (int k = 0; k < 4; ++k) rgba[k] = C[4 * (n - 1) + k]; return; }
  int i = 0;
  while (i < n - 2 && x >= P[i + 1]) ++i;
  double f = (x - P[i]) / (P[i + 1] - P[i]);
  for (int k = 0; k < 4; ++k) rgba[k] = (1.0 - f) * C[4 * i + k] + f * C[4 * (i + 1) + k];
}

/* Reading (camera, paper silent): pinhole camera, pixel centres, row 0 at the
 * top, right = normalize(f x up), up' = right x f, aspect W/H. */
void orc_camera_ray(const orc_camera* cam, int W, int H, int px, int py, double o[3], double d[3]) {
  double f[3], r[3], u[3];
  for (int a = 0; a < 3; ++a) f[a] = cam->target[a] - cam->eye[a];
  double nf = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (int a = 0; a < 3; ++a) f[a] /= nf;
  r[0] = f[1] * cam->up[2] - f[2] * cam->up[1];
  r[1] = f[2] * cam->up[0] - f[0] * cam->up[2];
  r[2] = f[0] * cam->up[1] - f[1] * cam->up[0];
  double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int a = 0; a < 3; ++a) r[a] /= nr;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  double th = tan(0.5 * cam->fovy);
  double sx = (2.0 * (px + 0.5) / W - 1.0) * th * ((double)W / (double)H);
  double sy = (1.0 - 2.0 * (py + 0.5) / H) * th;
  for (int a = 0; a < 3; ++a) d[a] = f[a] + sx * r[a] + sy * u[a];
  double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int a = 0; a < 3; ++a) { d[a] /= nd; o[a] = cam->eye[a]; }
}

/* Reading: the volume occupies the box [-0.5,0.5]^3 in world space; returns
 * 0 when the ray misses or the entry is not before the exit (tie = miss). */
int orc_box_intersect(const double o[3], const double d[3], double* t0, double* t1) {
  double tn = -INFINITY, tf = INFINITY;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0) {
      if (o[a] < -0.5 || o[a] > 0.5) return 0;
      continue;
    }
    double ta = (-0.5 - o[a]) / d[a], tb = (0.5 - o[a]) / d[a];
    if (ta > tb) { double s = ta; ta = tb; tb = s; }
    if (ta > tn) tn = ta;
    if (tb < tf) tf = tb;
  }
  *t0 = tn > 0.0 ? tn : 0.0;
  *t1 = tf;
  return *t1 > *t0;
}

/* Blinn-Phong with a headlight (Section 5: the gradient is the isosurface
 * normal used for Phong lighting).  Reading: n = -grad/|grad|, L = V = H = -d,
 * two-sided, rgb' = rgb (0.1 + 0.6 |n.L|) + 0.3 |n.H|^32, unshaded when
 * |grad| < 1e-6. */
static void shade(const double rgb[3], const double grad[3], const double d[3], double out[3]) {
  double g = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
  if (g < 1e-6) { out[0] = rgb[0]; out[1] = rgb[1]; out[2] = rgb[2]; return; }
  double c = fabs(grad[0] * d[0] + grad[1] * d[1] + grad[2] * d[2]) / g;
  double diff = 0.1 + 0.6 * c;
  double spec = 0.3 * pow(c, 32.0);
  for (int k = 0; k < 3; ++k) out[k] = rgb[k] * diff + spec;
}

/* Density sources the ray marcher can sample. */
typedef struct {
  const orc_net* net;   /* fV-SRN network, or NULL for the dense volume */
  const double* vol;    /* dense volume [z][y][x] */
  int nx, ny, nz;
  double time;
  int shading;
  double fd_h;          /* central-difference step (network coordinates) */
} orc_field;

static double field_density(const orc_field* fd, const double p[3], orc_trace* tr) {
  if (fd->net) { forward(fd->net, p, fd->time, tr); return tr->v[fd->net->l][0]; }
  double r;
  orc_trilinear(fd->vol, fd->nx, fd->ny, fd->nz, 1, p, &r);
  return r;
}

/* Central differences of the trilinear volume with a step of one voxel per
 * axis (h = 1 / (n_a - 1) along axis a), positions clamped to the domain
 * (Section 5 "FD"): the gradient of dense-grid shading and of the head's
 * training targets. */
void orc_volume_fd_grad(const double* vol, int nx, int ny, int nz, const double p[3], double g[3]) {
  int dims[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    double h = 1.0 / (double)(dims[a] - 1);
    double pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
    pp[a] = clamp01(p[a] + h);
    pm[a] = clamp01(p[a] - h);
    double vp, vm;
    orc_trilinear(vol, nx, ny, nz, 1, pp, &vp);
    orc_trilinear(vol, nx, ny, nz, 1, pm, &vm);
    g[a] = (vp - vm) / (2.0 * h);
  }
}

/* Precision model of a kernel path, for the first-order rounding-error
 * bounds that set the test tolerances of gradients and shaded images (see
 * the section "First-order rounding-error bounds" below; not the method). */
typedef struct {
  double in_rel, in_abs;   /* layer-0 inputs: |dv| <= in_rel |v| + in_abs */
  double act_abs, act_rel; /* hidden activations: |da| <= act_abs (1 + |x|) + act_rel |a| */
  double acc;              /* accumulation: |dx| <= acc K sum |terms| for the K terms of a layer */
  double dact_abs;         /* activation derivatives: |da'| <= dact_abs (1 + |x|) */
  double bwd_rel;          /* backward: relative error of each stored adjoint entry */
  double jac_rel;          /* Jacobian d v0 / d p: relative error of each term */
  double vol_abs;          /* dense volume samples: |drho| <= vol_abs */
  double lat_w;            /* latent weights rounded: |dz_c| += lat_w sum_k w_k |G_kc| */
} orc_prec;

static double sample_shade_bound(const orc_field* fd, const orc_prec* pr, const orc_trace* tr, const double p[3],
                                 const double grad[3], const double rgb[3], const double d[3]);

/* Ray march of one pixel (Section 3 DVR; Section 6: constant step).
 * Reading: segments [t0 + k ds, min(t0 + (k+1) ds, t1)], density sampled at
 * the segment midpoint, alpha = 1 - exp(-kappa * length), premultiplied
 * front-to-back compositing over black, terminated after the sample that
 * brings the opacity to et or above.  *margin receives min_k |A_k - et|. */
static void march(const orc_field* fd, const orc_tf* tf, const double o[3], const double d[3], double ds, double et,
                  double out[4], double* margin, long long* n_samples, orc_trace* tr, const orc_prec* pr,
                  double* bound) {
  if (bound) *bound = 0.0;
  double C[3] = {0, 0, 0}, A = 0.0, mg = INFINITY;
  long long ns = 0;
  double t0, t1;
  if (orc_box_intersect(o, d, &t0, &t1)) {
    for (long long k = 0;; ++k) {
      double ta = t0 + (double)k * ds;
      if (ta >= t1) break;
      double tb = t0 + (double)(k + 1) * ds;
      if (tb > t1) tb = t1;
      double len = tb - ta, tm = 0.5 * (ta + tb);
      double p[3];
      for (int a = 0; a < 3; ++a) p[a] = clamp01(o[a] + tm * d[a] + 0.5);
      double rho, grad[3] = {0, 0, 0};
      if (fd->net && fd->shading == ORC_SHADE_ADJOINT) {
        forward(fd->net, p, fd->time, tr);
        rho = tr->v[fd->net->l][0];
        input_grad_traced(fd->net, tr, fd->time, grad);
      } else if (fd->net && fd->shading == ORC_SHADE_HEAD) {
        forward(fd->net, p, fd->time, tr);
        rho = tr->v[fd->net->l][0];
        for (int a = 0; a < 3; ++a) grad[a] = tr->v[fd->net->l][1 + a];
      } else {
        rho = field_density(fd, p, tr);
        if (fd->shading == ORC_SHADE_FD && !fd->net) {
          /* dense volume: central differences, step of one voxel */
          orc_volume_fd_grad(fd->vol, fd->nx, fd->ny, fd->nz, p, grad);
        } else if (fd->shading == ORC_SHADE_FD) {
          /* network: central differences with the given step (Section 5 "FD") */
          for (int a = 0; a < 3; ++a) {
            double h = fd->fd_h;
            double pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
            pp[a] = clamp01(p[a] + h);
            pm[a] = clamp01(p[a] - h);
            grad[a] = (field_density(fd, pp, tr) - field_density(fd, pm, tr)) / (2.0 * h);
          }
        }
      }
      ++ns;
      double rgba[4];
      orc_tf_eval(tf, rho, rgba);
      double kappa = rgba[3] * tf->opacity_scale;
      double alpha = 1.0 - exp(-kappa * len);
      double rgb[3] = {rgba[0], rgba[1], rgba[2]};
      if (fd->shading != ORC_SHADE_NONE) shade(rgba, grad, d, rgb);
      double wgt = (1.0 - A) * alpha;
      if (bound && fd->shading != ORC_SHADE_NONE) {
        /* tolerance bookkeeping only: the composite weight times the bound
         * on the sample's shaded colour error */
        double rgb0[3] = {rgba[0], rgba[1], rgba[2]};
        if (fd->net && fd->shading == ORC_SHADE_FD) forward(fd->net, p, fd->time, tr);
        *bound += wgt * sample_shade_bound(fd, pr, tr, p, grad, rgb0, d);
      }
      for (int c = 0; c < 3; ++c) C[c] += wgt * rgb[c];
      A += wgt;
      double dm = fabs(A - et);
      if (dm < mg) mg = dm;
      if (A >= et) break;
    }
  }
  out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = A;
  if (margin) *margin = mg;
  if (n_samples) *n_samples = ns;
}

/* Pixel p of the batch [n_times][n_views][H][W] rendered into out[4*k] for
 * k-th listed pixel.  pix == NULL renders every pixel in order. */
static void render_common(const orc_net* net, const double* vol, int nx, int ny, int nz, const orc_camera* cams,
                          int n_views, const double* times, int n_times, const orc_tf* tf, int W, int H, double ds,
                          double et, int shading, double fd_h, const long long* pix, long long n_pix, double* out,
                          double* margin, long long* samples, const orc_prec* pr, double* bound) {
  long long total = pix ? n_pix : (long long)n_times * n_views * H * W;
  long long ns_sum = 0;
  #pragma omp parallel for schedule(dynamic, 16) reduction(+ : ns_sum)
  for (long long k = 0; k < total; ++k) {
    long long g = pix ? pix[k] : k;
    int px = (int)(g % W);
    int py = (int)((g / W) % H);
    int v = (int)((g / ((long long)W * H)) % n_views);
    int ti = (int)(g / ((long long)W * H * n_views));
    orc_field fd = {net, vol, nx, ny, nz, times ? times[ti] : 0.0, shading, fd_h};
    double o[3], d[3];
    orc_camera_ray(&cams[v], W, H, px, py, o, d);
    orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
    long long ns = 0;
    march(&fd, tf, o, d, ds, et, out + 4 * k, margin ? margin + k : NULL, &ns, tr, pr, bound ? bound + k : NULL);
    free(tr);
    ns_sum += ns;
  }
  if (samples) *samples = ns_sum;
}

/* fV-SRN render (network evaluated at every sample). */
void orc_render(const orc_net* net, const orc_camera* cams, int n_views, const double* times, int n_times,
                const orc_tf* tf, int W, int H, double ds, double et, int shading, double fd_h, const long long* pix,
                long long n_pix, double* out, double* margin, long long* samples) {
  render_common(net, NULL, 0, 0, 0, cams, n_views, times, n_times, tf, W, H, ds, et, shading, fd_h, pix, n_pix, out,
                margin, samples, NULL, NULL);
}

/* orc_render plus, per pixel, the first-order bound on the image error that
 * the gradient error of a kernel path with precision model prec (an array of
 * the orc_prec fields in order) causes through the shading (test
 * tolerances; see "First-order rounding-error bounds"). */
void orc_render_shade_bound(const orc_net* net, const orc_camera* cams, int n_views, const double* times, int n_times,
                            const orc_tf* tf, int W, int H, double ds, double et, int shading, double fd_h,
                            const long long* pix, long long n_pix, const double* prec, double* out, double* bound) {
  orc_prec pr;
  memcpy(&pr, prec, sizeof(pr));
  render_common(net, NULL, 0, 0, 0, cams, n_views, times, n_times, tf, W, H, ds, et, shading, fd_h, pix, n_pix, out,
                NULL, NULL, &pr, bound);
}

/* Dense-grid DVR of the raw volume (the reference renderer of Section 4). */
void orc_dvr_dense(const double* vol, int nx, int ny, int nz, const orc_camera* cams, int n_views, const orc_tf* tf,
                   int W, int H, double ds, double et, int shading, const long long* pix, long long n_pix,
                   double* out, double* margin, long long* samples) {
  render_common(NULL, vol, nx, ny, nz, cams, n_views, NULL, 1, tf, W, H, ds, et, shading, 0.0, pix, n_pix, out,
                margin, samples, NULL, NULL);
}

/* orc_dvr_dense plus the per-pixel shading error bound (FD shading, volume
 * samples off by at most prec.vol_abs). */
void orc_dvr_dense_shade_bound(const double* vol, int nx, int ny, int nz, const orc_camera* cams, int n_views,
                               const orc_tf* tf, int W, int H, double ds, double et, const long long* pix,
                               long long n_pix, const double* prec, double* out, double* bound) {
  orc_prec pr;
  memcpy(&pr, prec, sizeof(pr));
  render_common(NULL, vol, nx, ny, nz, cams, n_views, NULL, 1, tf, W, H, ds, et, ORC_SHADE_FD, 0.0, pix, n_pix, out,
                NULL, NULL, &pr, bound);
}

/* ------------------------------------------------------------------------ */
static double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

/* ------------------------------------------------------------------------ */
/* Section 6.2 adaptive resampling.  Every N fit steps the prediction error is
 * estimated on a coarse voxel grid E (res^3 voxels, paper: 128^3) from a few
 * positions per voxel (paper: 8), and the next steps draw their training
 * points with counts proportional to E.
 *
 * Position i of voxel v = (vx, vy, vz) (v = (vz res + vy) res + vx):
 * Philox4x32-10 of counter (v, i, 0x4552, 0), key (seed low, seed high);
 * u_a = (word_a >> 8) 2^-24 and p_a = (v_a + u_a) / res, both operations in
 * FP32 round-to-nearest (the position is an input both implementations
 * derive identically).  Reading: the error is the L1 error of output 0 (the
 * density) against the trilinear volume, the loss of the fit. */
static float orc_voxel_coord(int va, uint32_t word, int res) {
  float u = (float)(word >> 8) * (1.0f / 16777216.0f);
  volatile float s = (float)va + u; /* one FP32 rounding, no contraction */
  return s / (float)res;
}

void orc_error_grid(const orc_net* n, const double* vol, int nx, int ny, int nz, int res, int spv, uint64_t seed,
                    double t, double* E) {
  size_t nvox = (size_t)res * res * res;
  orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (size_t v = 0; v < nvox; ++v) {
    int vx = (int)(v % res), vy = (int)((v / res) % res), vz = (int)(v / ((size_t)res * res));
    double acc = 0.0;
    for (int i = 0; i < spv; ++i) {
      uint32_t ctr[4] = {(uint32_t)v, (uint32_t)i, 0x4552u, 0u}, o[4];
      orc_philox4x32_10(ctr, key, o);
      double p[3] = {orc_voxel_coord(vx, o[0], res), orc_voxel_coord(vy, o[1], res), orc_voxel_coord(vz, o[2], res)};
      double y;
      orc_trilinear(vol, nx, ny, nz, 1, p, &y);
      forward(n, p, t, tr);
      acc += fabs(tr->v[n->l][0] - y);
    }
    E[v] = acc / (double)spv;
  }
  free(tr);
}

/* Integer sampling distribution from an error grid (given as the FP32 values
 * the GPU holds): q_v = floor(E_v * (65535 / max E)) in FP32, clamped to
 * [0, 65535]; S is the exclusive prefix sum of q (S[0] = 0, S[nvox] = Q).
 * Returns 0, or 1 when an entry is negative or not finite.  Q = 0 (a zero
 * grid) means uniform sampling. */
int orc_adaptive_cdf(const float* E, int res, uint64_t* S) {
  size_t nvox = (size_t)res * res * res;
  float mx = 0.0f;
  for (size_t v = 0; v < nvox; ++v) {
    if (!isfinite(E[v]) || E[v] < 0.0f) return 1;
    if (E[v] > mx) mx = E[v];
  }
  S[0] = 0;
  volatile float scale = mx > 0.0f ? 65535.0f / mx : 0.0f;
  for (size_t v = 0; v < nvox; ++v) {
    volatile float x = E[v] * scale;
    float f = floorf(x);
    uint32_t q = f >= 65535.0f ? 65535u : (uint32_t)f;
    S[v + 1] = S[v] + q;
  }
  return 0;
}

/* Point j of n for fit step `step` under the distribution S: the voxel holds
 * the stratum midpoint t_j = floor((2j + 1) Q / (2n)), i.e. the voxel v with
 * S[v] <= t_j < S[v + 1] (so voxel v receives round(n q_v / Q) points, +-1);
 * the offset inside it uses the uniform sampler's Philox draw (counter
 * (j, step, 0x5352, 0)).  Requires (2n + 1) Q < 2^64. */
void orc_adaptive_point(const uint64_t* S, int res, uint64_t seed, int step, int j, int n, double p[3]) {
  size_t nvox = (size_t)res * res * res;
  uint64_t Q = S[nvox];
  uint64_t tj = ((uint64_t)(2 * (uint64_t)j + 1) * Q) / (2 * (uint64_t)n);
  size_t lo = 0, hi = nvox; /* S[lo] <= tj < S[hi] */
  while (hi - lo > 1) {
    size_t mid = (lo + hi) / 2;
    if (S[mid] <= tj) lo = mid; else hi = mid;
  }
  int vx = (int)(lo % res), vy = (int)((lo / res) % res), vz = (int)(lo / ((size_t)res * res));
  uint32_t ctr[4] = {(uint32_t)j, (uint32_t)step, 0x5352u, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  p[0] = orc_voxel_coord(vx, o[0], res);
  p[1] = orc_voxel_coord(vy, o[1], res);
  p[2] = orc_voxel_coord(vz, o[2], res);
}

/* The training point j of a fit step: uniform (S == NULL or Q == 0) or
 * adaptive. */
static void fit_point(const uint64_t* S, int res, uint64_t seed, int step, int j, int n, double p[3]) {
  if (S && S[(size_t)res * res * res] > 0) orc_adaptive_point(S, res, seed, step, j, n, p);
  else orc_sample_point(seed, step, j, p);
}

/* Loss and parameter gradients of one fit step without the update.
 * Section 5 world-space training: L1 loss between the prediction and the
 * trilinear ground truth at uniformly drawn points.  Reading for the 4-output
 * head (loss in the paper's missing supplement): L = mean_j(|rho_j - y_j|
 * + gw * sum_a |g_ja - gs * dV_a(p_j)|), dV by central differences.
 * The time of every point is t (one frame).  Gradients are overwritten.
 * cdf (may be NULL): the Section 6.2 adaptive distribution of
 * orc_adaptive_cdf over cdf_res^3 voxels. */
double orc_fit_loss_grad(const orc_net* n, const double* vol, int nx, int ny, int nz, int n_points, uint64_t seed,
                         int step, double t, double gw, double gs, double* dW, double* db, double* dgrid,
                         const uint64_t* cdf, int cdf_res) {
  size_t nW = 0, nb = 0;
  for (int i = 0; i < n->l; ++i) { nW += (size_t)layer_out(n, i) * layer_in(n, i); nb += layer_out(n, i); }
  size_t ng = (size_t)n->nkey * n->R * n->R * n->R * n->F;
  memset(dW, 0, nW * sizeof(double));
  memset(db, 0, nb * sizeof(double));
  memset(dgrid, 0, ng * sizeof(double));
  orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
  double loss = 0.0;
  double inv_n = 1.0 / (double)n_points;
  for (int j = 0; j < n_points; ++j) {
    double p[3];
    fit_point(cdf, cdf_res, seed, step, j, n_points, p);
    double y;
    orc_trilinear(vol, nx, ny, nz, 1, p, &y);
    forward(n, p, t, tr);
    double dout[ORC_MAXW];
    for (int d = 0; d < n->D; ++d) dout[d] = 0.0;
    double r = tr->v[n->l][0] - y;
    loss += fabs(r);
    dout[0] = sgn(r) * inv_n;
    if (n->D == 4) {
      double gv[3];
      orc_volume_fd_grad(vol, nx, ny, nz, p, gv);
      for (int a = 0; a < 3; ++a) {
        double ra = tr->v[n->l][1 + a] - gs * gv[a];
        loss += gw * fabs(ra);
        dout[1 + a] = gw * sgn(ra) * inv_n;
      }
    }
    backward(n, tr, t, dout, dW, db, dgrid, NULL);
  }
  free(tr);
  return loss * inv_n;
}

/* The density residuals r_j = rho(p_j) - y_j of a fit step's points (the
 * quantity whose sign the L1 gradient takes) and the points themselves
 * (n_points x 3): test infrastructure for deciding which points' signs are
 * settled beyond rounding. */
void orc_fit_residuals(const orc_net* n, const double* vol, int nx, int ny, int nz, int n_points, uint64_t seed,
                       int step, double t, const uint64_t* cdf, int cdf_res, double* r, double* pts) {
  #pragma omp parallel for schedule(dynamic, 256)
  for (int j = 0; j < n_points; ++j) {
    orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
    double* p = pts + 3 * (size_t)j;
    fit_point(cdf, cdf_res, seed, step, j, n_points, p);
    double y;
    orc_trilinear(vol, nx, ny, nz, 1, p, &y);
    forward(n, p, t, tr);
    r[j] = tr->v[n->l][0] - y;
    free(tr);
  }
}

/* Adam (Kingma & Ba 2015) with bias correction at step index step+1.
 * Reading: beta1 0.9, beta2 0.999, eps 1e-8 (paper names Adam, lr 0.01). */
void orc_adam(double* theta, double* m, double* v, const double* g, size_t n, double lr, int step, double beta1,
              double beta2, double eps) {
  double bc1 = 1.0 - pow(beta1, step + 1), bc2 = 1.0 - pow(beta2, step + 1);
  for (size_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    double mh = m[i] / bc1, vh = v[i] / bc2;
    theta[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* One full fit step: loss, gradients, Adam on grid (lr_grid) and on W, b
 * (lr_net).  adam_m / adam_v are packed [grid | W | b].  Returns the loss;
 * when the loss or a gradient is not finite the parameters are left
 * unchanged and *status is set to 1. */
double orc_fit_step(orc_net* n, double* adam_m, double* adam_v, const double* vol, int nx, int ny, int nz,
                    int n_points, uint64_t seed, int step, double t, double lr_grid, double lr_net, double gw,
                    double gs, double* grads_out, int* status, const uint64_t* cdf, int cdf_res) {
  size_t nW = 0, nb = 0;
  for (int i = 0; i < n->l; ++i) { nW += (size_t)layer_out(n, i) * layer_in(n, i); nb += layer_out(n, i); }
  size_t ng = (size_t)n->nkey * n->R * n->R * n->R * n->F;
  double* g = (double*)malloc(sizeof(double) * (ng + nW + nb));
  double loss = orc_fit_loss_grad(n, vol, nx, ny, nz, n_points, seed, step, t, gw, gs, g + ng, g + ng + nW, g, cdf,
                                  cdf_res);
  int finite = isfinite(loss);
  for (size_t i = 0; i < ng + nW + nb && finite; ++i) finite = isfinite(g[i]);
  if (grads_out) memcpy(grads_out, g, sizeof(double) * (ng + nW + nb));
  if (!finite) { *status = 1; free(g); return loss; }
  *status = 0;
  orc_adam(n->grid, adam_m, adam_v, g, ng, lr_grid, step, 0.9, 0.999, 1e-8);
  orc_adam(n->W, adam_m + ng, adam_v + ng, g + ng, nW, lr_net, step, 0.9, 0.999, 1e-8);
  orc_adam(n->b, adam_m + ng + nW, adam_v + ng + nW, g + ng + nW, nb, lr_net, step, 0.9, 0.999, 1e-8);
  free(g);
  return loss;
}

/* ------------------------------------------------------------------------ */
/* Section 6.2 "off" baseline: the volume low-pass filtered and resampled to a
 * grid of the latent grid's memory.  Reading: separable Gaussian with
 * sigma = 0.5 (N-1)/(M-1) voxels, truncated at 3 sigma, clamp-to-edge, then
 * vertex-aligned trilinear resampling to M^3. */
void orc_lowpass_resample(const double* vol, int nx, int ny, int nz, int M, double* out) {
  int dims[3] = {nx, ny, nz};
  size_t nvox = (size_t)nx * ny * nz;
  double* a = (double*)malloc(sizeof(double) * nvox);
  double* b = (double*)malloc(sizeof(double) * nvox);
  memcpy(a, vol, sizeof(double) * nvox);
  for (int ax = 0; ax < 3; ++ax) {
    double sigma = 0.5 * (double)(dims[ax] - 1) / (double)(M - 1);
    int rad = (int)ceil(3.0 * sigma);
    double* w = (double*)malloc(sizeof(double) * (2 * rad + 1));
    double ws = 0.0;
    for (int k = -rad; k <= rad; ++k) { w[k + rad] = exp(-0.5 * k * k / (sigma * sigma)); ws += w[k + rad]; }
    for (int k = 0; k <= 2 * rad; ++k) w[k] /= ws;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          double s = 0.0;
          for (int k = -rad; k <= rad; ++k) {
            int c[3] = {x, y, z};
            c[ax] += k;
            if (c[ax] < 0) c[ax] = 0;
            if (c[ax] > dims[ax] - 1) c[ax] = dims[ax] - 1;
            s += w[k + rad] * a[((size_t)c[2] * ny + c[1]) * nx + c[0]];
          }
          b[((size_t)z * ny + y) * nx + x] = s;
        }
    double* t = a; a = b; b = t;
    free(w);
  }
  for (int z = 0; z < M; ++z)
    for (int y = 0; y < M; ++y)
      for (int x = 0; x < M; ++x) {
        double p[3] = {(double)x / (M - 1), (double)y / (M - 1), (double)z / (M - 1)};
        orc_trilinear(a, nx, ny, nz, 1, p, &out[((size_t)z * M + y) * M + x]);
      }
  free(a);
  free(b);
}

/* Image PSNR over the RGB channels of n RGBA pixels (peak 1). */
double orc_psnr(const double* a, const double* b, long long n) {
  double se = 0.0;
  for (long long i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) { double d = a[4 * i + c] - b[4 * i + c]; se += d * d; }
  double mse = se / (3.0 * (double)n);
  return mse == 0.0 ? INFINITY : 10.0 * log10(1.0 / mse);
}

/* SSIM (Wang, Bovik, Sheikh, Simoncelli 2004): 11x11 Gaussian window with
 * sigma 1.5, K1 0.01, K2 0.03, dynamic range 1, windows fully inside the
 * image, mean over the RGB channels of H x W RGBA images. */
double orc_ssim(const double* a, const double* b, int W, int H) {
  double w[11], ws = 0.0;
  for (int k = 0; k < 11; ++k) { w[k] = exp(-0.5 * (k - 5) * (k - 5) / (1.5 * 1.5)); ws += w[k]; }
  for (int k = 0; k < 11; ++k) w[k] /= ws;
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
  double total = 0.0;
  long long cnt = 0;
  for (int c = 0; c < 3; ++c)
    for (int y = 5; y < H - 5; ++y)
      for (int x = 5; x < W - 5; ++x) {
        double mx = 0, my = 0, sxx = 0, syy = 0, sxy = 0;
        for (int j = -5; j <= 5; ++j)
          for (int i = -5; i <= 5; ++i) {
            double ww = w[j + 5] * w[i + 5];
            double va = a[4 * ((size_t)(y + j) * W + (x + i)) + c];
            double vb = b[4 * ((size_t)(y + j) * W + (x + i)) + c];
            mx += ww * va; my += ww * vb;
            sxx += ww * va * va; syy += ww * vb * vb; sxy += ww * va * vb;
          }
        sxx -= mx * mx; syy -= my * my; sxy -= mx * my;
        total += ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2));
        ++cnt;
      }
  return cnt ? total / (double)cnt : 1.0;
}

/* ------------------------------------------------------------------------ */
/* First-order rounding-error bounds (test infrastructure: they set the
 * tolerances of the gradient and shaded-image tests; the method does not use
 * them).  A kernel path is described by an orc_prec: how far each layer-0
 * input, hidden activation, accumulated sum, activation derivative, adjoint
 * entry and Jacobian term may be off.  Every such rounding site s is off by
 * at most c_s |d y / d site_s| in its effect on an output y, to first order.
 * The sites are distinct rounding operations; modelled as independent,
 * mean-zero and bounded (the probabilistic model of Higham and Mary, "A new
 * approach to probabilistic rounding error analysis", SIAM J. Sci. Comput.
 * 41, 2019), Hoeffding's inequality bounds the total by
 * lambda sqrt(sum_s c_s^2) except with probability 2 exp(-lambda^2 / 2);
 * lambda = 6 makes that 3e-8 per bounded quantity.  An inner product of K
 * terms contributes one site of scale acc sqrt(K) sum |terms| (the same
 * paper's bound for a length-K sum).  Sensitivities of outputs are one
 * backward pass; those of the adjoint gradient to the forward pass are
 * central differences of the traced gradient with respect to each
 * pre-activation, and to the backward pass the linear maps from each
 * adjoint entry to the gradient. */
#define ORC_LAMBDA 6.0

/* delta[i][o] = d out_d / d h_i[o] for every layer i of a traced evaluation. */
static void layer_deltas(const orc_net* n, const orc_trace* tr, int d, double delta[ORC_MAXL][ORC_MAXW]) {
  size_t woff[ORC_MAXL + 1];
  woff[0] = 0;
  for (int i = 0; i < n->l; ++i) woff[i + 1] = woff[i] + (size_t)layer_out(n, i) * layer_in(n, i);
  for (int o = 0; o < n->D; ++o) delta[n->l - 1][o] = (o == d) ? 1.0 : 0.0;
  for (int i = n->l - 1; i >= 1; --i) {
    int din = layer_in(n, i), dout_i = layer_out(n, i);
    const double* W = n->W + woff[i];
    for (int j = 0; j < din; ++j) {
      double g = 0.0;
      for (int o = 0; o < dout_i; ++o) g += W[(size_t)o * din + j] * delta[i][o];
      delta[i - 1][j] = g * act_df(n->act, tr->h[i - 1][j]);
    }
  }
}

/* sum_k w_k |G_kc| over the 8 corners (and the two keyframes, with their
 * time weights) of the trilinear latent vector at the traced position. */
static void latent_abs(const orc_net* n, const orc_trace* tr, double t, double* za) {
  size_t gsz = (size_t)n->R * n->R * n->R * n->F;
  int k0, ix, iy, iz;
  double f, fx, fy, fz;
  time_weights(n, t, &k0, &f);
  cell_coord(tr->p[0], n->R, &ix, &fx);
  cell_coord(tr->p[1], n->R, &iy, &fy);
  cell_coord(tr->p[2], n->R, &iz, &fz);
  for (int c = 0; c < n->F; ++c) za[c] = 0.0;
  for (int kk = 0; kk < (n->nkey > 1 ? 2 : 1); ++kk) {
    double tw = (n->nkey > 1) ? (kk ? f : 1.0 - f) : 1.0;
    const double* G = n->grid + (size_t)(k0 + kk) * gsz;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          double w = tw * (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
          size_t v = (((size_t)(iz + dz) * n->R + (iy + dy)) * n->R + (ix + dx)) * (size_t)n->F;
          for (int c = 0; c < n->F; ++c) za[c] += w * fabs(G[v + c]);
        }
  }
}

/* Scales of the forward sites: sv[i][j] for input j of layer i (its
 * rounding), sr[i][o] for the accumulation of pre-activation h_i[o]. */
static void forward_sites(const orc_net* n, const orc_trace* tr, double t, const orc_prec* pr,
                          double sv[ORC_MAXL][ORC_MAXW], double sr[ORC_MAXL][ORC_MAXW]) {
  const double* W = n->W;
  const double* b = n->b;
  double za[ORC_MAXW];
  if (pr->lat_w > 0.0) latent_abs(n, tr, t, za);
  for (int i = 0; i < n->l; ++i) {
    int din = layer_in(n, i), dout_i = layer_out(n, i);
    int K = i == 0 ? din + 2 : 2 * din + 2;
    for (int j = 0; j < din; ++j) {
      double v = tr->v[i][j];
      sv[i][j] = i == 0 ? pr->in_rel * fabs(v) + pr->in_abs
                        : pr->act_abs * (1.0 + fabs(tr->h[i - 1][j])) + pr->act_rel * fabs(v);
      int zc = j - 3 - 2 * n->m;
      if (i == 0 && pr->lat_w > 0.0 && zc >= 0 && zc < n->F) sv[i][j] += pr->lat_w * za[zc];
    }
    for (int o = 0; o < dout_i; ++o) {
      double mag = fabs(b[o]);
      for (int j = 0; j < din; ++j) mag += fabs(W[(size_t)o * din + j] * tr->v[i][j]);
      sr[i][o] = pr->acc * sqrt((double)K) * mag;
    }
    W += (size_t)dout_i * din;
    b += dout_i;
  }
}

/* Bound on the error of output d of a traced evaluation. */
static double output_bound(const orc_net* n, const orc_trace* tr, double t, const orc_prec* pr, int d) {
  static __thread double sv[ORC_MAXL][ORC_MAXW], sr[ORC_MAXL][ORC_MAXW], delta[ORC_MAXL][ORC_MAXW];
  forward_sites(n, tr, t, pr, sv, sr);
  layer_deltas(n, tr, d, delta);
  double var = 0.0;
  const double* W = n->W;
  for (int i = 0; i < n->l; ++i) {
    int din = layer_in(n, i), dout_i = layer_out(n, i);
    for (int j = 0; j < din; ++j) {
      double dj = 0.0; /* d out_d / d v_i[j] */
      for (int o = 0; o < dout_i; ++o) dj += delta[i][o] * W[(size_t)o * din + j];
      var += dj * dj * sv[i][j] * sv[i][j];
    }
    for (int o = 0; o < dout_i; ++o) var += delta[i][o] * delta[i][o] * sr[i][o] * sr[i][o];
    W += (size_t)dout_i * din;
  }
  return ORC_LAMBDA * sqrt(var);
}

/* Jacobian d v0 / d p (d0 x 3) at the traced position. */
static void input_jacobian(const orc_net* n, const orc_trace* tr, double t, double* J) {
  int d0 = layer_in(n, 0);
  memset(J, 0, sizeof(double) * 3 * d0);
  for (int a = 0; a < 3; ++a) J[3 * a + a] = 1.0;
  for (int k = 0; k < n->m; ++k)
    for (int a = 0; a < 3; ++a) {
      J[3 * (3 + k) + a] = cos(tr->e[k]) * n->fourier[3 * k + a];
      J[3 * (3 + n->m + k) + a] = -sin(tr->e[k]) * n->fourier[3 * k + a];
    }
  size_t gsz = (size_t)n->R * n->R * n->R * n->F;
  int k0;
  double f;
  time_weights(n, t, &k0, &f);
  double jac[3 * ORC_MAXW];
  for (int kk = 0; kk < (n->nkey > 1 ? 2 : 1); ++kk) {
    double tw = (n->nkey > 1) ? (kk ? f : 1.0 - f) : 1.0;
    orc_trilinear_grad(n->grid + (size_t)(k0 + kk) * gsz, n->R, n->R, n->R, n->F, tr->p, jac);
    for (int ch = 0; ch < n->F; ++ch)
      for (int a = 0; a < 3; ++a) J[3 * (3 + 2 * n->m + ch) + a] += tw * jac[3 * ch + a];
  }
}

/* Layers after layer i of a trace recomputed after h_i changed. */
static void forward_from(const orc_net* n, orc_trace* tr, int i) {
  const double* W = n->W;
  const double* b = n->b;
  for (int q = 0; q < n->l; ++q) {
    int din = layer_in(n, q), dout_q = layer_out(n, q);
    if (q == i) {
      for (int o = 0; o < dout_q; ++o) tr->v[q + 1][o] = (q < n->l - 1) ? act_f(n->act, tr->h[q][o]) : tr->h[q][o];
    } else if (q > i) {
      for (int o = 0; o < dout_q; ++o) {
        double h = b[o];
        for (int j = 0; j < din; ++j) h += W[(size_t)o * din + j] * tr->v[q][j];
        tr->h[q][o] = h;
        tr->v[q + 1][o] = (q < n->l - 1) ? act_f(n->act, h) : h;
      }
    }
    W += (size_t)dout_q * din;
    b += dout_q;
  }
}

/* g = J^T W0^T delta_0, the adjoint gradient of output 0, of a trace (J
 * fixed: the kernels evaluate the Jacobian at the sample position). */
static void traced_gradient(const orc_net* n, const orc_trace* tr, const double* J, double g[3],
                            double delta[ORC_MAXL][ORC_MAXW], double* dv0) {
  layer_deltas(n, tr, 0, delta);
  int d0 = layer_in(n, 0), c0 = layer_out(n, 0);
  for (int j = 0; j < d0; ++j) {
    double s = 0.0;
    for (int o = 0; o < c0; ++o) s += n->W[(size_t)o * d0 + j] * delta[0][o];
    dv0[j] = s;
  }
  for (int a = 0; a < 3; ++a) {
    g[a] = 0.0;
    for (int j = 0; j < d0; ++j) g[a] += J[3 * j + a] * dv0[j];
  }
}

/* Bound (per component) on the error of the adjoint gradient of output 0. */
static void gradient_bound(const orc_net* n, const orc_trace* tr0, double t, const orc_prec* pr, double B[3]) {
  static __thread double sv[ORC_MAXL][ORC_MAXW], sr[ORC_MAXL][ORC_MAXW], delta[ORC_MAXL][ORC_MAXW];
  static __thread double dl2[ORC_MAXL][ORC_MAXW], S[ORC_MAXL][ORC_MAXW][3];
  static __thread double J[3 * ORC_MAXW], dv0[ORC_MAXW], dv1[ORC_MAXW], M[3][ORC_MAXW], M2[3][ORC_MAXW];
  static __thread orc_trace tr;
  int d0 = layer_in(n, 0), c = n->c, L = n->l;
  size_t woff[ORC_MAXL + 1];
  woff[0] = 0;
  for (int i = 0; i < L; ++i) woff[i + 1] = woff[i] + (size_t)layer_out(n, i) * layer_in(n, i);
  forward_sites(n, tr0, t, pr, sv, sr);
  input_jacobian(n, tr0, t, J);
  double g0[3], var[3] = {0.0, 0.0, 0.0};
  traced_gradient(n, tr0, J, g0, delta, dv0);
  /* forward sites: S[i][o] = d g / d h_i[o] by central differences (the
   * linear output layer does not enter the gradient) */
  for (int i = 0; i < L - 1; ++i)
    for (int o = 0; o < c; ++o) {
      double eta = 1e-6 * (1.0 + fabs(tr0->h[i][o])), gp[3], gm[3];
      memcpy(&tr, tr0, sizeof(tr));
      tr.h[i][o] += eta;
      forward_from(n, &tr, i);
      traced_gradient(n, &tr, J, gp, dl2, dv1);
      memcpy(&tr, tr0, sizeof(tr));
      tr.h[i][o] -= eta;
      forward_from(n, &tr, i);
      traced_gradient(n, &tr, J, gm, dl2, dv1);
      for (int a = 0; a < 3; ++a) S[i][o][a] = (gp[a] - gm[a]) / (2.0 * eta);
    }
  for (int i = 0; i < L - 1; ++i) {
    const double* W = n->W + woff[i];
    int din = layer_in(n, i);
    for (int j = 0; j < din; ++j)
      for (int a = 0; a < 3; ++a) {
        double s = 0.0; /* d g_a / d v_i[j] */
        for (int o = 0; o < c; ++o) s += S[i][o][a] * W[(size_t)o * din + j];
        var[a] += s * s * sv[i][j] * sv[i][j];
      }
    for (int o = 0; o < c; ++o)
      for (int a = 0; a < 3; ++a) var[a] += S[i][o][a] * S[i][o][a] * sr[i][o] * sr[i][o];
  }
  /* backward sites.  M (3 x c) maps a change of delta_i to the gradient:
   * M_0 = J^T W0^T, M_{i+1} = M_i diag(a'(h_i)) W_{i+1}^T.  Each adjoint
   * entry delta_i[j] = (W_{i+1}^T delta_{i+1})_j a'(h_i[j]) carries: its
   * storage (bwd_rel |delta|), the derivative (|(W^T delta)_j| dact
   * (1 + |h|)) and the accumulation (acc sqrt(2c) sum_o |W_oj delta_o|
   * |a'|); the final dv0 accumulation and the Jacobian terms enter through J
   * directly. */
  for (int a = 0; a < 3; ++a)
    for (int o = 0; o < c; ++o) {
      double s = 0.0;
      for (int j = 0; j < d0; ++j) s += J[3 * j + a] * n->W[(size_t)o * d0 + j];
      M[a][o] = s;
    }
  for (int i = 0; i <= L - 2; ++i) {
    const double* Wn = n->W + woff[i + 1]; /* layer i+1: rows o' (its outputs), columns j (= h_i entries) */
    int dn = layer_out(n, i + 1);
    for (int j = 0; j < c; ++j) {
      double gsum = 0.0, mag = 0.0;
      for (int o2 = 0; o2 < dn; ++o2) {
        double w = Wn[(size_t)o2 * c + j], dd = (i + 1 == L - 1) ? (o2 == 0 ? 1.0 : 0.0) : delta[i + 1][o2];
        gsum += w * dd;
        mag += fabs(w * dd);
      }
      double ad = act_df(n->act, tr0->h[i][j]);
      double e_store = pr->bwd_rel * fabs(delta[i][j]);
      double e_der = fabs(gsum) * pr->dact_abs * (1.0 + fabs(tr0->h[i][j]));
      double e_acc = (i + 1 == L - 1) ? 0.0 : pr->acc * sqrt((double)(2 * c)) * mag * fabs(ad);
      for (int a = 0; a < 3; ++a) {
        double m = M[a][j];
        var[a] += m * m * (e_store * e_store + e_der * e_der + e_acc * e_acc);
      }
    }
    if (i + 1 <= L - 2) { /* M_{i+1} = M_i diag(a'(h_i)) W_{i+1}^T */
      for (int a = 0; a < 3; ++a)
        for (int o2 = 0; o2 < c; ++o2) {
          double s = 0.0;
          for (int j = 0; j < c; ++j) s += M[a][j] * act_df(n->act, tr0->h[i][j]) * Wn[(size_t)o2 * c + j];
          M2[a][o2] = s;
        }
      memcpy(M, M2, sizeof(M));
    }
  }
  for (int j = 0; j < d0; ++j) {
    double mag = 0.0;
    for (int o = 0; o < c; ++o) mag += fabs(n->W[(size_t)o * d0 + j] * delta[0][o]);
    double e_acc = pr->acc * sqrt((double)(2 * c)) * mag;
    for (int a = 0; a < 3; ++a) {
      double ej = J[3 * j + a] * e_acc, ejac = pr->jac_rel * J[3 * j + a] * dv0[j];
      var[a] += ej * ej + ejac * ejac;
    }
  }
  for (int a = 0; a < 3; ++a) B[a] = ORC_LAMBDA * sqrt(var[a]);
}

/* Per point: bounds on the error of every output (n_pts x D) and of the
 * adjoint gradient of output 0 (n_pts x 3, may be NULL), for a kernel path
 * with precision model prec (the orc_prec fields in order). */
void orc_error_bounds(const orc_net* n, const double* pts, int n_pts, double t, const double* prec, double* B_out,
                      double* B_grad) {
  orc_prec pr;
  memcpy(&pr, prec, sizeof(pr));
  #pragma omp parallel for schedule(dynamic, 16)
  for (int j = 0; j < n_pts; ++j) {
    orc_trace* tr = (orc_trace*)malloc(sizeof(orc_trace));
    forward(n, pts + 3 * j, t, tr);
    for (int d = 0; d < n->D; ++d) B_out[(size_t)j * n->D + d] = output_bound(n, tr, t, &pr, d);
    if (B_grad) gradient_bound(n, tr, t, &pr, B_grad + 3 * (size_t)j);
    free(tr);
  }
}

/* The shaded colour of one sample is rgb (0.1 + 0.6 c) + 0.3 c^32 with
 * c = |n.d| (the reading of Section 5's Phong shading); a gradient error e
 * moves the unit normal by at most 2 e / |g|, so c by at most
 * min(1, 2 e / |g|), and the colour by (0.6 max rgb + 9.6 c^31) times that
 * (to first order).  A sample whose |g| lies within e of the 1e-6 unshaded
 * threshold may switch between shaded and unshaded: up to 0.9 max rgb + 0.3.
 * e per mode: the adjoint's gradient bound; for central differences the
 * density bounds of the two neighbours over 2h per axis; for the head the
 * bounds of outputs 1..3. */
static double sample_shade_bound(const orc_field* fd, const orc_prec* pr, const orc_trace* tr, const double p[3],
                                 const double grad[3], const double rgb[3], const double d[3]) {
  double e2 = 0.0;
  if (fd->net && fd->shading == ORC_SHADE_ADJOINT) {
    double B[3];
    gradient_bound(fd->net, tr, fd->time, pr, B);
    e2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  } else if (fd->net && fd->shading == ORC_SHADE_HEAD) {
    for (int a = 0; a < 3; ++a) {
      double b = output_bound(fd->net, tr, fd->time, pr, 1 + a);
      e2 += b * b;
    }
  } else if (fd->shading == ORC_SHADE_FD) {
    orc_trace* tq = (orc_trace*)malloc(sizeof(orc_trace));
    for (int a = 0; a < 3; ++a) {
      double h = fd->net ? fd->fd_h : 1.0 / (double)((a == 0 ? fd->nx : a == 1 ? fd->ny : fd->nz) - 1);
      double s = 0.0;
      for (int sg = -1; sg <= 1; sg += 2) {
        double q[3] = {p[0], p[1], p[2]};
        q[a] = clamp01(p[a] + sg * h);
        if (fd->net) {
          forward(fd->net, q, fd->time, tq);
          s += output_bound(fd->net, tq, fd->time, pr, 0);
        } else {
          s += pr->vol_abs;
        }
      }
      e2 += (s / (2.0 * h)) * (s / (2.0 * h));
    }
    free(tq);
  }
  double e = sqrt(e2);
  double gn = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
  double mrgb = fmax(rgb[0], fmax(rgb[1], rgb[2]));
  double bound = 0.0;
  if (gn - e < 1e-6) bound += 0.9 * mrgb + 0.3; /* may switch between shaded and unshaded */
  if (gn >= 1e-6) {
    double c = fabs(grad[0] * d[0] + grad[1] * d[1] + grad[2] * d[2]) / gn;
    double dc = fmin(1.0, 2.0 * e / gn);
    double cmax = fmin(1.0, c + dc);
    bound += (0.6 * mrgb + 9.6 * pow(cmax, 31.0)) * dc;
  }
  return bound;
}
