"""Shared helpers of the GPU parity tests: build a network on both sides from
the same seeded inputs, run the CUDA path through the C ABI and the FP64
oracle, and compare."""
import math

import numpy as np

import oracle
from paper_2112_01579_gb300 import synth

# Tolerances (stated in the test plan): FP32 CUDA-core path 1e-5 image
# max-abs and 1e-5 relative density; FP16 tensor-core path 2e-3 image
# max-abs and 1e-3 relative density.  Relative density error is
# |d rho| / max(|rho_ref|, 1) since volumes are normalised to [0, 1].
TOL_FP32_IMG = 1e-5
TOL_FP32_RHO = 1e-5
TOL_FP16_IMG = 2e-3
TOL_FP16_RHO = 1e-3
# Pixels whose oracle opacity came within ET_BAND of the termination
# threshold may terminate one sample apart on the two sides; the composite
# then differs by at most (1 - et) * max colour.
ET_BAND = 1e-3
TOL_ET_FLIP = 1e-2


def oracle_tf(tf):
    return oracle.OracleTF(tf["pos"], tf["rgba"], tf["opacity_scale"])


def rel_density_err(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)


def compare_images(got, ref, margin, tol, et):
    """Max-abs comparison with the early-termination rule; tol is a number
    or one bound per pixel.  Returns a dict (max_strict / worst_ratio: the
    largest error and error / bound over the strictly compared pixels)."""
    got = np.asarray(got, np.float64).reshape(-1, 4)
    ref = np.asarray(ref, np.float64).reshape(-1, 4)
    err = np.abs(got - ref).max(axis=1)
    tol = np.broadcast_to(np.asarray(tol, np.float64).reshape(-1), err.shape)
    if et <= 1.0 and margin is not None:
        near = np.asarray(margin).reshape(-1) < ET_BAND
    else:
        near = np.zeros(len(err), bool)
    strict = ~near
    flip = np.maximum(tol, TOL_ET_FLIP)
    return dict(max_strict=float(err[strict].max()) if strict.any() else 0.0,
                worst_ratio=float((err[strict] / tol[strict]).max()) if strict.any() else 0.0,
                max_near=float(err[near].max()) if near.any() else 0.0, n_near=int(near.sum()),
                ok=bool(np.all(err[strict] <= tol[strict]) and np.all(err[near] <= flip[near])))


def shaded_tol(img_tol, bound):
    """Per-pixel bound of a shaded image: the unshaded image bound plus the
    bound on what the gradient error of the path moves through the shading
    (oracle.render_shade_bound)."""
    return img_tol + np.asarray(bound, np.float64)


def dense_sample_error(vol):
    """Bound on the FP32 dense-DVR density error at a sample: the FP32
    trilinear interpolation (a few roundings of values <= max |V|, 2^-21 max
    |V|) and the sample position's FP32 rounding (rays and steps in FP32,
    2^-20 absolute) times the largest slope of the volume."""
    v = np.asarray(vol, np.float64)
    slope = max(float(np.abs(np.diff(v, axis=a)).max()) * (v.shape[a] - 1) for a in range(3))
    return 2.0 ** -21 * float(np.abs(v).max()) + 2.0 ** -20 * slope


def cfg1_params(seed=0):
    """Config 1 network: 8^3 x 8 FP32 latent grid N(0, 0.01^2) (here wider so
    the latent term matters), 4 Fourier frequencies (m = 12), 2 layers of
    width 32, sine, Xavier weights."""
    return synth.random_params(R=8, F=8, m=12, layers=2, width=32, out_dim=1, act=synth.ACT_SINE, seed=seed,
                               grid_std=0.5, bias_std=0.2)


def cfg2_params(seed=0, R=32, out_dim=1, nkey=1, key_times=None):
    """Config 2 network: 32^3 x 16 latent grid, m = 14, 4 layers of width
    32, SnakeAlt."""
    return synth.random_params(R=R, F=16, m=14, layers=4, width=32, out_dim=out_dim, act=synth.ACT_SNAKEALT,
                               seed=seed, grid_std=0.5, bias_std=0.2, n_keyframes=nkey, key_times=key_times)


# ---------------------------------------------------------------- L1 fit signs
def tc_fit_forward_bound(p):
    """Bound on |rho_gpu - y_gpu - (rho - y)| of the tensor-core fit's
    forward (two-layer width-32 network, Section 5 world-space fit), summed
    over every error source at its worst:
    * layer-0 inputs: NeRF Fourier features by one MUFU sin / cos per axis
      (absolute error 2^-20.9 each, so 2^-20.4 as a complex rotation) and angle
      doubling, which doubles that error per octave: row k (octave k div 3)
      is off by 2^(k div 3 - 20.4) + 2^-22; other Fourier matrices use the
      compensated sin / cos (2^-21); the latent vector is an FP32 trilinear
      of grid values (2^-21 max |grid|); positions are exact;
    * every input and weight enters as FP16 hi + lo (2^-21 relative per
      product) and the tensor cores accumulate 3 (d0 + 2) products in FP32
      (2^-24 each, worst case: K 2^-24 sum |terms|);
    * the activation: 2^-20 (1 + |x|); the FP32 output sum over 33 terms;
      the FP32 trilinear target (2^-22)."""
    W0, W1 = [np.abs(np.asarray(w, np.float64)) for w in p["weights"]]
    b0, b1 = [np.abs(np.asarray(b, np.float64)) for b in p["biases"]]
    F0 = np.asarray(p["fourier"], np.float64)
    m = F0.shape[0]
    nerf = np.array_equal(np.asarray(p["fourier"], np.float32), synth.nerf_fourier_matrix(m))
    gmax = max(1.0, float(np.abs(p["grid"]).max()))
    F = np.asarray(p["grid"]).shape[-1]
    d0 = W0.shape[1]
    feat = np.array([2.0 ** (k // 3 - 20.4) + 2.0 ** -22 if nerf else 2.0 ** -21 for k in range(m)])
    eps_v = np.concatenate([np.zeros(3), feat, feat, np.full(F, 2.0 ** -21 * gmax), np.zeros(d0 - 3 - 2 * m - F)])
    vmax = np.concatenate([np.ones(3 + 2 * m), np.full(F, gmax), np.ones(d0 - 3 - 2 * m - F)])
    mag = W0 @ vmax + b0
    pre = W0 @ eps_v + (2.0 ** -21 + 3 * (d0 + 2) * 2.0 ** -24) * mag
    act = pre + 2.0 ** -20 * (1.0 + mag)
    return float((W1[0] * act).sum() + 33 * 2.0 ** -24 * (W1[0].sum() + b1[0]) + 2.0 ** -22)
def _flat_grad(dW, db, dg):
    return np.concatenate([np.asarray(dg).ravel(), np.concatenate([w.ravel() for w in dW]), np.concatenate(db)])


def l1_fit_gradient_check(g_gpu, p, vol, n, seed, step, tol, t=0.0, cdf=None):
    """The GPU's L1-loss gradient of one fit step (flat [grid | W | b])
    against the oracle's, with the one freedom L1 leaves (several results are
    correct): a point whose oracle residual r_j lies within the forward error
    bound eps of zero may take either sign (or zero) on the GPU.  Those
    points' oracle contributions sign(r_j) P_j / n (P_j = d rho / d theta at
    p_j) are replaced by s_j P_j / n, s_j in {-1, 0, 1} fitted by least
    squares to the GPU gradient; every entry must then agree within tol of
    its block's maximum.  Returns (loss, g_oracle, per-entry uncertainty,
    number of undecided points, number whose sign the GPU took differently)."""
    on = oracle.OracleNet(p)
    r, P = oracle.fit_residuals(on, vol, n, seed, step, t, cdf=cdf)
    eps = tc_fit_forward_bound(p)
    amb = np.flatnonzero(np.abs(r) <= eps)
    lo, dW, db, dg = oracle.fit_loss_grad(on, vol, n, seed, step, t, cdf=cdf)
    g_orc = _flat_grad(dW, db, dg)
    ng, nW = on.grid.size, on.W.size
    blocks = [slice(0, ng), slice(ng, ng + nW), slice(ng + nW, g_orc.size)]
    want = g_orc.copy()
    unc = np.zeros_like(g_orc)
    flips = 0
    if amb.size:
        Pj = []
        for j in amb:
            w, b, g = oracle.net_backward(on, P[j:j + 1], np.ones((1, on.dims["D"])), t)
            Pj.append(_flat_grad(w, b, g))
        Pj = np.stack(Pj, axis=1)  # [n_params, n_amb]
        excl = g_orc - Pj @ (np.sign(r[amb]) / n)
        coef, *_ = np.linalg.lstsq(Pj, (np.asarray(g_gpu, np.float64) - excl) * n, rcond=None)
        s = np.clip(np.rint(coef), -1, 1)
        want = excl + Pj @ (s / n)
        flips = int(np.sum(s != np.sign(r[amb])))
        unc = np.abs(Pj).sum(axis=1) * (2.0 / n)
    for sl in blocks:
        scale = max(np.abs(g_orc[sl]).max(), 1e-30)
        err = np.abs(np.asarray(g_gpu, np.float64)[sl] - want[sl]).max() / scale
        assert err <= tol, (sl, err, amb.size, flips)
        unc[sl] += tol * scale
    return lo, g_orc, unc, int(amb.size), flips


def quantize_u8(grid, F):
    """The 8-bit latent-grid rule stated in srn.h, in float32 like the
    device: per channel over all keyframes and vertices lo = min, step =
    (max - lo) / 255 (1 when max == lo), code = round((g - lo) / step)."""
    g = np.asarray(grid, np.float32).reshape(-1, F)
    lo = g.min(axis=0)
    hi = g.max(axis=0)
    step = np.where(hi > lo, (hi - lo) / np.float32(255.0), np.float32(1.0)).astype(np.float32)
    code = np.clip(np.rint((g - lo[None]) / step[None]), 0, 255).astype(np.uint8)
    return code.reshape(-1), lo, step


def u8_params(params):
    """The parameters as the FP16 path reads them with the 8-bit grid: the
    dequantized grid lo + step * code (computed here from the stated rule;
    the device's codes are tested bit-exact against it)."""
    q = dict(params)
    g = np.asarray(params["grid"], np.float32)
    F = g.shape[-1]
    code, lo, step = quantize_u8(g, F)
    deq = lo[None].astype(np.float64) + step[None].astype(np.float64) * code.reshape(-1, F).astype(np.float64)
    q["grid"] = deq.reshape(g.shape)
    return q


def oracle_trained_params(vol, p, steps=60, n=4096, seed=9, lr_grid=1e-2, lr_net=5e-3):
    """A network trained by the oracle's own fit (FP64 Adam on the L1 loss),
    rounded to FP16: weights and grid moved away from their initial ranges
    without any value from the CUDA path."""
    on = oracle.OracleNet(p)
    n_par = on.grid.size + on.W.size + on.b.size
    m, v = np.zeros(n_par), np.zeros(n_par)
    for s in range(steps):
        oracle.fit_step(on, m, v, vol, n, seed, s, lr_grid, lr_net)
    q = dict(p)
    q["grid"] = on.grid.reshape(np.asarray(p["grid"]).shape).astype(np.float32)
    q["weights"] = [w.astype(np.float32) for w in on.unpack_W(on.W)]
    q["biases"] = [b.astype(np.float32) for b in on.unpack_b(on.b)]
    return synth.to_half_exact(q)
