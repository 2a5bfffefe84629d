"""Seeded synthetic inputs for the fV-SRN render / fit path.

This module holds no arithmetic of the method itself: it only produces inputs
(volumes, initial parameters, the Fourier matrix, transfer functions, cameras)
that both the GPU path and the CPU oracle consume.  The paper's datasets
(ScalarFlow, Ejecta, RM, Skull, Jet) are not available; these seeded volumes
stand in for them with the same sizes and kinds of structure:

* ``blobs_volume``: a sum of isotropic Gaussian blobs (smooth, sparse).
* ``noise_volume``: fractal gradient noise (Perlin's improved noise, SIGGRAPH
  2002, summed over octaves), dense fine-scale detail like turbulent smoke.
* ``aniso_blobs_volume``: rotated anisotropic blobs plus a little noise
  (surface-like structure for shaded rendering).
* ``moving_blobs_volumes``: blobs translating linearly in time (time series).

Volumes are float32 ``[nz, ny, nx]`` with x fastest, sampled at the grid
vertices ``x / (n - 1)`` of the unit cube, normalised to [0, 1].  Large
volumes can be produced on a CUDA device (``device="cuda"``); the blob and
noise parameters come from numpy's seeded generator either way.
"""
from __future__ import annotations

import math

import numpy as np

ACT_SINE, ACT_SNAKEALT = 0, 1


def _torch():
    import torch
    return torch


def _coords(n, device, dtype):
    torch = _torch()
    return torch.linspace(0.0, 1.0, n, device=device, dtype=dtype)


def _normalise(v):
    lo, hi = v.min(), v.max()
    return (v - lo) / (hi - lo) if float(hi - lo) > 0 else v * 0


def blobs_volume(n=64, n_blobs=8, seed=0, device="cpu", sigma=(0.05, 0.15), amp=(0.3, 1.0)):
    """Sum of isotropic Gaussians, centres U[0,1]^3, sigma and amplitude
    uniform in the given ranges, min-max normalised to [0,1]."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, 1, (n_blobs, 3))
    s = rng.uniform(*sigma, n_blobs)
    a = rng.uniform(*amp, n_blobs)
    x = _coords(n, device, torch.float64)
    v = torch.zeros((n, n, n), device=device, dtype=torch.float64)
    for k in range(n_blobs):
        gx = torch.exp(-0.5 * ((x - c[k, 0]) / s[k]) ** 2)
        gy = torch.exp(-0.5 * ((x - c[k, 1]) / s[k]) ** 2)
        gz = torch.exp(-0.5 * ((x - c[k, 2]) / s[k]) ** 2)
        v += a[k] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return _normalise(v).to(torch.float32)


_GRAD12 = np.array([[1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0], [1, 0, 1], [-1, 0, 1], [1, 0, -1],
                    [-1, 0, -1], [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1]], dtype=np.float64)


def _gradient_noise(x, y, z, perm, grads):
    """Perlin gradient noise at coordinates x, y, z (tensors of one shape):
    lattice gradients picked by a hashed permutation, quintic fade."""
    torch = _torch()
    xi, yi, zi = torch.floor(x), torch.floor(y), torch.floor(z)
    fx, fy, fz = x - xi, y - yi, z - zi
    X, Y, Z = xi.long() & 255, yi.long() & 255, zi.long() & 255

    def fade(t):
        return t * t * t * (t * (t * 6 - 15) + 10)

    u, v, w = fade(fx), fade(fy), fade(fz)

    def corner(dx, dy, dz):
        h = perm[perm[perm[X + dx] + Y + dy] + Z + dz] % 12
        g = grads[h]
        return g[..., 0] * (fx - dx) + g[..., 1] * (fy - dy) + g[..., 2] * (fz - dz)

    def lerp(a, b, t):
        return a + t * (b - a)

    x00 = lerp(corner(0, 0, 0), corner(1, 0, 0), u)
    x10 = lerp(corner(0, 1, 0), corner(1, 1, 0), u)
    x01 = lerp(corner(0, 0, 1), corner(1, 0, 1), u)
    x11 = lerp(corner(0, 1, 1), corner(1, 1, 1), u)
    return lerp(lerp(x00, x10, v), lerp(x01, x11, v), w)


def _noise_raw(n, octaves, base_freq, gain, lacunarity, seed, device):
    torch = _torch()
    rng = np.random.default_rng(seed)
    p = rng.permutation(256)
    perm = torch.as_tensor(np.concatenate([p, p, p]), device=device)
    grads = torch.as_tensor(_GRAD12, device=device, dtype=torch.float32)
    offs = rng.uniform(0, 64, (octaves, 3))
    x = _coords(n, device, torch.float32)
    out = torch.zeros((n, n, n), device=device, dtype=torch.float32)
    for o in range(octaves):
        f = base_freq * lacunarity ** o
        for zc in range(0, n, 64):  # slab-wise to bound temporaries
            zz = x[zc:zc + 64]
            Z, Y, X = torch.meshgrid(zz * f + offs[o, 2], x * f + offs[o, 1], x * f + offs[o, 0], indexing="ij")
            out[zc:zc + 64] += (gain ** o) * _gradient_noise(X, Y, Z, perm, grads)
    return out


def noise_volume(n=256, octaves=5, base_freq=4.0, gain=0.5, lacunarity=2.0, seed=0, device="cpu"):
    """Fractal gradient noise: sum over octaves of noise at base_freq *
    lacunarity^o with weight gain^o, min-max normalised to [0,1]."""
    return _normalise(_noise_raw(n, octaves, base_freq, gain, lacunarity, seed, device))


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def aniso_blobs_volume(n=512, n_blobs=64, seed=0, noise_amp=0.1, device="cpu"):
    """Rotated anisotropic Gaussians (axis sigma U[0.02,0.12], amplitude
    U[0.3,1]) plus noise_amp times fractal noise, min-max normalised."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    x = _coords(n, device, torch.float32)
    out = torch.zeros((n, n, n), device=device, dtype=torch.float32)
    blobs = []
    for _ in range(n_blobs):
        c = rng.uniform(0.1, 0.9, 3)
        s = rng.uniform(0.02, 0.12, 3)
        a = rng.uniform(0.3, 1.0)
        R = _rotation(rng)
        Q = R @ np.diag(1.0 / s ** 2) @ R.T  # precision matrix
        blobs.append((c, Q, a, 4.0 * s.max()))
    for zc in range(0, n, 32):
        zz = x[zc:zc + 32]
        Z, Y, X = torch.meshgrid(zz, x, x, indexing="ij")
        for c, Q, a, rad in blobs:
            dx, dy, dz = X - c[0], Y - c[1], Z - c[2]
            q = (Q[0, 0] * dx * dx + Q[1, 1] * dy * dy + Q[2, 2] * dz * dz
                 + 2 * (Q[0, 1] * dx * dy + Q[0, 2] * dx * dz + Q[1, 2] * dy * dz))
            out[zc:zc + 32] += a * torch.exp(-0.5 * q)
    out = _normalise(out)
    if noise_amp:
        out = out + noise_amp * _normalise(_noise_raw(n, 5, 4.0, 0.5, 2.0, seed + 1, device))
    return _normalise(out)


def moving_blobs_volumes(n=256, n_steps=16, n_blobs=32, seed=0, device="cpu"):
    """n_steps frames of blobs with centres c0 + v t / (n_steps - 1),
    v U[-0.2,0.2]^3, sigma U[0.05,0.15]; one global min-max over all frames.
    Returns a float32 tensor [n_steps, n, n, n]."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    c0 = rng.uniform(0.2, 0.8, (n_blobs, 3))
    vel = rng.uniform(-0.2, 0.2, (n_blobs, 3))
    s = rng.uniform(0.05, 0.15, n_blobs)
    a = rng.uniform(0.3, 1.0, n_blobs)
    x = _coords(n, device, torch.float32)
    out = torch.zeros((n_steps, n, n, n), device=device, dtype=torch.float32)
    for t in range(n_steps):
        c = c0 + vel * t / max(n_steps - 1, 1)
        for k in range(n_blobs):
            gx = torch.exp(-0.5 * ((x - c[k, 0]) / s[k]) ** 2)
            gy = torch.exp(-0.5 * ((x - c[k, 1]) / s[k]) ** 2)
            gz = torch.exp(-0.5 * ((x - c[k, 2]) / s[k]) ** 2)
            out[t] += a[k] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return _normalise(out)


# --------------------------------------------------------------------------
def nerf_fourier_matrix(m: int) -> np.ndarray:
    """The fixed NeRF Fourier matrix (row k = 2 pi 2^(k // 3) e_(k mod 3)),
    truncated to m rows when m is not a multiple of 3."""
    F = np.zeros((m, 3), dtype=np.float32)
    for k in range(m):
        F[k, k % 3] = 2.0 * math.pi * (2.0 ** (k // 3))
    return F


def fourier_rows_for_width(width: int, F: int = 16) -> int:
    """Fourier rows m for hidden width c in the width sweep: the input vector
    3 + 2m + F plus one padding column is c + 16 wide, as the 48-column
    input of the 32-channel network (Section 4.2 figure) is."""
    m2 = width + 16 - 1 - 3 - F
    if m2 <= 0 or m2 % 2:
        raise ValueError("no Fourier count fits this width")
    return m2 // 2


def layer_dims(F, m, layers, width, out_dim, time_input=0):
    d = [3 + 2 * m + F + time_input] + [width] * (layers - 1) + [out_dim]
    return list(zip(d[:-1], d[1:]))


def init_params(R=8, F=8, m=12, layers=2, width=32, out_dim=1, act=ACT_SINE, n_keyframes=1, seed=0,
                grid_std=0.01, key_times=None, time_input=0):
    """Initial parameters: Xavier-uniform weights, zero biases, latent grid
    N(0, grid_std^2), NeRF Fourier matrix.  All float32 numpy arrays.
    time_input = 1 adds the time as one more network input."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for din, dout in layer_dims(F, m, layers, width, out_dim, time_input):
        a = math.sqrt(6.0 / (din + dout))
        Ws.append(rng.uniform(-a, a, (dout, din)).astype(np.float32))
        bs.append(np.zeros(dout, dtype=np.float32))
    grid = rng.normal(0.0, grid_std, (n_keyframes, R, R, R, F)).astype(np.float32)
    if key_times is None:
        key_times = np.arange(n_keyframes, dtype=np.float32)
    return dict(grid=grid, fourier=nerf_fourier_matrix(m), weights=Ws, biases=bs, act=act,
                key_times=np.asarray(key_times, dtype=np.float32), time_input=int(time_input))


def random_params(R=8, F=8, m=12, layers=2, width=32, out_dim=1, act=ACT_SINE, n_keyframes=1, seed=0,
                  grid_std=0.5, w_gain=1.0, bias_std=0.1, key_times=None, time_input=0):
    """Like init_params but with a latent grid and biases large enough that
    every term of the network matters (used by parity tests)."""
    p = init_params(R, F, m, layers, width, out_dim, act, n_keyframes, seed, grid_std, key_times, time_input)
    rng = np.random.default_rng(seed + 7919)
    p["weights"] = [(w * w_gain).astype(np.float32) for w in p["weights"]]
    p["biases"] = [rng.normal(0, bias_std, b.shape).astype(np.float32) for b in p["biases"]]
    return p


def to_half_exact(params):
    """Round weights, biases and grid to float16 and back to float32, so that
    FP16 storage on the GPU and the oracle's FP64 copy hold identical values."""
    q = dict(params)
    q["grid"] = params["grid"].astype(np.float16).astype(np.float32)
    q["weights"] = [w.astype(np.float16).astype(np.float32) for w in params["weights"]]
    q["biases"] = [b.astype(np.float16).astype(np.float32) for b in params["biases"]]
    return q


# --------------------------------------------------------------------------
def tf_preset(n_points: int, opacity_scale: float = 20.0):
    """Piecewise-linear RGBA transfer functions with 4 or 8 control points."""
    if n_points == 4:
        pos = [0.0, 0.35, 0.65, 1.0]
        rgba = [[0.0, 0.0, 0.0, 0.0], [0.2, 0.4, 1.0, 0.05], [1.0, 0.6, 0.2, 0.4], [1.0, 1.0, 1.0, 1.0]]
    elif n_points == 8:
        pos = [0.0, 0.2, 0.3, 0.4, 0.55, 0.7, 0.85, 1.0]
        rgba = [[0.0, 0.0, 0.0, 0.0], [0.1, 0.2, 0.9, 0.0], [0.2, 0.5, 1.0, 0.15], [0.3, 0.9, 0.6, 0.02],
                [0.9, 0.9, 0.2, 0.3], [1.0, 0.5, 0.1, 0.05], [1.0, 0.2, 0.1, 0.6], [1.0, 1.0, 1.0, 1.0]]
    else:
        raise ValueError("presets exist for 4 and 8 points")
    return dict(pos=np.asarray(pos, np.float32), rgba=np.asarray(rgba, np.float32),
                opacity_scale=float(opacity_scale))


def orbit_cameras(n_views=8, radius=1.0, elevation_deg=20.0, fovy_deg=90.0, az0_deg=22.5):
    """Cameras on a sphere looking at the origin: azimuth az0 + 360 k / n."""
    cams = []
    el = math.radians(elevation_deg)
    for k in range(n_views):
        az = math.radians(az0_deg + 360.0 * k / n_views)
        eye = [radius * math.cos(el) * math.cos(az), radius * math.sin(el), radius * math.cos(el) * math.sin(az)]
        cams.append(dict(eye=eye, target=[0.0, 0.0, 0.0], up=[0.0, 1.0, 0.0], fovy=math.radians(fovy_deg)))
    return cams


def sample_pixels(T, V, H, W, n, seed=0):
    """n distinct flat pixel indices of a [T, V, H, W] batch (sorted)."""
    rng = np.random.default_rng(seed)
    total = T * V * H * W
    n = min(n, total)
    return np.sort(rng.choice(total, size=n, replace=False)).astype(np.int64)
