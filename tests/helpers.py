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
    """Max-abs comparison with the early-termination rule; returns a dict."""
    got = np.asarray(got, np.float64).reshape(-1, 4)
    ref = np.asarray(ref, np.float64).reshape(-1, 4)
    err = np.abs(got - ref).max(axis=1)
    if et <= 1.0 and margin is not None:
        near = np.asarray(margin).reshape(-1) < ET_BAND
    else:
        near = np.zeros(len(err), bool)
    strict = err[~near]
    return dict(max_strict=float(strict.max()) if strict.size else 0.0,
                max_near=float(err[near].max()) if near.any() else 0.0, n_near=int(near.sum()),
                ok=bool((strict.size == 0 or strict.max() <= tol) and (not near.any() or err[near].max() <= TOL_ET_FLIP)))


def conditioned_tol(render, tol, delta=2.0 ** -23):
    """FP32 image tolerance that accounts for the conditioning of the image.

    The FP32 kernels compute camera rays and sample positions in FP32, so a
    sample position carries a rounding error of a few units of 2^-24.  For
    networks with high Fourier octaves (or large inputs such as a raw time
    value) the exact FP64 image already changes by more than the fixed
    tolerance when the camera moves by that much.  The tolerance returned is
    the larger of ``tol`` and twice the largest change of the oracle image
    when every camera eye moves by +-delta along (1, -1, 1).  ``render(cams)``
    renders with the given cameras (a list of camera dicts)."""
    import copy
    base = None
    worst = 0.0
    for sgn in (1.0, -1.0):
        cams = render.cameras
        shifted = copy.deepcopy(cams)
        for c in shifted:
            c["eye"] = [c["eye"][0] + sgn * delta, c["eye"][1] - sgn * delta, c["eye"][2] + sgn * delta]
        if base is None:
            base = np.asarray(render(cams), np.float64)
        worst = max(worst, float(np.abs(np.asarray(render(shifted), np.float64) - base).max()))
    return max(tol, 2.0 * worst)


class OracleRender:
    """Oracle render with fixed network, TF and image settings; called with
    a camera list (for conditioned_tol)."""

    def __init__(self, net, cams, tf, W, H, step, et, **kw):
        self.net, self.cameras, self.tf, self.args, self.kw = net, cams, tf, (W, H, step, et), kw

    def __call__(self, cams):
        return oracle.render(self.net, cams, oracle_tf(self.tf), *self.args, **self.kw)[0]


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
