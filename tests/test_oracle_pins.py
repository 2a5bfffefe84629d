"""More pins of the FP64 oracle against closed forms (no GPU).

* One-voxel central differences of a dense volume (Section 5 "FD": the
  dense-grid shading gradient and the head's training targets): exact on
  quadratic fields, per axis, on a volume with three different extents.
* The low-pass "off" baseline of Section 6.2: a cosine is attenuated by the
  Gaussian's transfer factor exp(-sigma^2 omega^2 / 2) for
  sigma = 0.5 (N - 1) / (M - 1) voxels along each axis.
* SSIM (Section 6 image quality; Wang et al. 2004): on ramps, the window's
  second moment enters the contrast term in closed form.
* Section 6.2 adaptive resampling: point counts per voxel proportional to
  the error E, within the bound the 16-bit weights allow.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2112_01579_gb300 import synth


def _quad(x, y, z):
    return 0.7 * x * x - 0.4 * y * y + 1.1 * z * z + 0.3 * x * y - 0.2 * y * z + 0.5 * x - 0.1


def _quad_grad(x, y, z):
    return np.array([1.4 * x + 0.3 * y + 0.5, -0.8 * y + 0.3 * x - 0.2 * z, 2.2 * z - 0.2 * y])


def _vertex_volume(f, nx, ny, nz):
    """f sampled at the vertices p_a = i / (n_a - 1); layout [z][y][x]."""
    z, y, x = np.meshgrid(np.linspace(0, 1, nz), np.linspace(0, 1, ny), np.linspace(0, 1, nx), indexing="ij")
    return f(x, y, z)


def test_volume_central_differences_exact_on_quadratics():
    """For a quadratic sampled at the vertices, the one-voxel central
    difference of the trilinear interpolant equals the exact derivative at
    every interior point: along axis a the two samples p +- h_a e_a sit at the
    same fraction of their cells, and (1-f)(q(i+1) - q(i-1)) + f(q(i+2) -
    q(i)) = 2 h q'(x) for a quadratic q.  With extents 9 x 13 x 17 the
    per-axis step 1/(n_a - 1) is the only one that gives the exact value
    (a step of 1/n_a, or another axis's step, leaves an O(h) error)."""
    nx, ny, nz = 9, 13, 17
    vol = _vertex_volume(_quad, nx, ny, nz)
    rng = np.random.default_rng(601)
    h = np.array([1 / (nx - 1), 1 / (ny - 1), 1 / (nz - 1)])
    for _ in range(200):
        p = h + rng.uniform(0, 1, 3) * (1 - 2 * h)  # p +- h stays inside [0, 1]
        g = oracle.volume_fd_grad(vol, p)
        np.testing.assert_allclose(g, _quad_grad(*p), rtol=0, atol=1e-12)
    # clamped at a face: the one-sided difference of the vertex values
    p = np.array([0.0, 0.5, 0.5])
    g = oracle.volume_fd_grad(vol, p)
    want = (_quad(h[0], 0.5, 0.5) - _quad(0.0, 0.5, 0.5)) / (2 * h[0])
    assert abs(g[0] - want) < 1e-12


def test_dense_fd_shading_uses_the_exact_gradient():
    """Dense DVR with FD shading of a field quadratic in x and y, constant in
    z, seen by a narrow camera on the z axis: every sample's p +- h stays
    inside the box along x and y (no clamping), so the shading gradient is
    the exact one and the image has a closed form (constant TF, so every
    segment's opacity depends only on its length)."""
    nx, ny, nz = 9, 13, 6

    def q(x, y, z):
        return 0.8 * (x - 0.5) ** 2 - 0.5 * (y - 0.5) ** 2 + 0.3 * (x - 0.5) * (y - 0.5) + 0.4 + 0 * z

    vol = _vertex_volume(q, nx, ny, nz)
    # FP32 values, as the C ABI passes them (the oracle widens them exactly)
    rgba = np.array([0.9, 0.6, 0.3, 0.1], np.float32).astype(np.float64)
    tf = oracle.OracleTF([0.0, 1.0], [rgba, rgba], 20.0)
    cam = dict(eye=[0.0, 0.0, 2.0], target=[0.0, 0.0, 0.0], up=[0.0, 1.0, 0.0],
               fovy=float(np.float32(math.radians(12.0))))
    W, H, ds = 7, 5, 1 / 32
    got, _, _ = oracle.dvr_dense(vol, [cam], tf, W, H, ds, 2.0, shading=oracle.SHADE_FD)
    kappa = rgba[3] * 20.0
    for py in range(H):
        for px in range(W):
            o, d = oracle.camera_ray(cam, W, H, px, py)
            hit, t0, t1 = oracle.box_intersect(o, d)
            assert hit
            C, A, k = np.zeros(3), 0.0, 0
            while t0 + k * ds < t1:
                ta, tb = t0 + k * ds, min(t0 + (k + 1) * ds, t1)
                p = np.clip(o + 0.5 * (ta + tb) * d + 0.5, 0, 1)
                assert 1 / (nx - 1) <= p[0] <= 1 - 1 / (nx - 1) and 1 / (ny - 1) <= p[1] <= 1 - 1 / (ny - 1)
                g = np.array([1.6 * (p[0] - 0.5) + 0.3 * (p[1] - 0.5), -1.0 * (p[1] - 0.5) + 0.3 * (p[0] - 0.5), 0.0])
                if np.linalg.norm(g) < 1e-6:  # the reading's unshaded case (the centre ray)
                    rgb = rgba[:3]
                else:
                    c = abs(g @ d) / np.linalg.norm(g)
                    rgb = rgba[:3] * (0.1 + 0.6 * c) + 0.3 * c ** 32
                a = 1 - math.exp(-kappa * (tb - ta))
                C += (1 - A) * a * rgb
                A += (1 - A) * a
                k += 1
            np.testing.assert_allclose(got[0, py, px], [*C, A], rtol=0, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_lowpass_attenuates_a_cosine_by_the_gaussian_transfer(axis):
    """Extents 33 x 17 x 65 resampled to M = 9 give sigma = 2, 1, 4 voxels
    along x, y, z, and output vertex j falls on source vertex r_a j (r = 4, 2,
    8), so no interpolation enters.  A cosine of period 8 sigma voxels along
    the tested axis (constant along the others, which the normalised filter
    keeps) comes out as H cos, H = exp(-sigma^2 omega^2 / 2), at vertices at
    least 3 sigma from the clamped borders.  The 3-sigma truncation and the
    sampling of the kernel move H by < 3e-3; sigma twice or half the stated
    value gives 0.29 or 0.93 instead of 0.73."""
    dims = (33, 17, 65)  # nx, ny, nz
    M = 9
    sigma = 0.5 * (dims[axis] - 1) / (M - 1)
    ratio = (dims[axis] - 1) // (M - 1)
    omega = 2 * math.pi / (8 * sigma)
    idx = np.arange(dims[axis], dtype=np.float64)
    shape = [1, 1, 1]
    shape[2 - axis] = dims[axis]
    vol = np.broadcast_to(np.cos(omega * idx).reshape(shape), dims[::-1]).copy()
    out = oracle.lowpass_resample(vol, M)
    H = math.exp(-0.5 * sigma ** 2 * omega ** 2)
    for j in range(M):
        src = ratio * j
        if src < 3 * sigma or src > dims[axis] - 1 - 3 * sigma:
            continue
        sl = [slice(None)] * 3
        sl[2 - axis] = j
        np.testing.assert_allclose(out[tuple(sl)], H * math.cos(omega * src), rtol=0, atol=3e-3)


def test_ssim_window_second_moment_on_ramps():
    """a = c + s x (R), c + s y (G), c + s (x + y) / 2 (B); b = lam a.  For a
    symmetric window of unit sum the local mean is the ramp's value at the
    window centre and the local variance is s^2 m2 (s^2 m2 / 2 for B), m2 the
    window's second moment along one axis (sigma^2 = 2.25 for the stated
    Gaussian; its 11-tap truncation gives 2.2435), so SSIM = mean over
    centres and channels of (2 lam mu^2 + C1) / ((1 + lam^2) mu^2 + C1) x
    (2 lam v + C2) / ((1 + lam^2) v + C2).  A window of sigma 1 or 2 moves the
    result by more than 1e-2."""
    Wd, Hd, c, s, lam = 48, 40, 0.2, 0.015, 0.6
    y, x = np.meshgrid(np.arange(Hd, dtype=np.float64), np.arange(Wd, dtype=np.float64), indexing="ij")
    a = np.zeros((Hd, Wd, 4))
    a[..., 0] = c + s * x
    a[..., 1] = c + s * y
    a[..., 2] = c + s * (x + y) / 2
    a[..., 3] = 1.0
    b = lam * a
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    m2 = 1.5 ** 2
    cy, cx = np.meshgrid(np.arange(5, Hd - 5, dtype=np.float64), np.arange(5, Wd - 5, dtype=np.float64),
                         indexing="ij")
    tot = 0.0
    for mu, v in ((c + s * cx, s * s * m2), (c + s * cy, s * s * m2), (c + s * (cx + cy) / 2, s * s * m2 / 2)):
        lum = (2 * lam * mu * mu + C1) / ((1 + lam * lam) * mu * mu + C1)
        cs = (2 * lam * v + C2) / ((1 + lam * lam) * v + C2)
        tot += (lum * cs).mean()
    want = tot / 3
    assert abs(oracle.ssim(a, b) - want) < 5e-4, (oracle.ssim(a, b), want)


def _voxel_of(pts, res):
    v = np.floor(np.asarray(pts) * res).astype(int).clip(0, res - 1)
    return (v[:, 2] * res + v[:, 1]) * res + v[:, 0]


def test_adaptive_counts_proportional_to_the_error():
    """Section 6.2: voxel v receives a number of points proportional to its
    error E_v.  Against the exact proportional count n E_v / sum E (FP64),
    the 16-bit weights q_v = floor(65535 E_v / max E) allow a deviation of at
    most 1 + n (1 + nvox e_v / sum e) * 1.004 / Q, e_v = 65535 E_v / max E,
    Q >= sum e - 1.004 nvox (the floor loses < 1 per voxel, the FP32 product
    < 0.004).  Independent draws would miss this by sqrt(n E_v / sum E)."""
    res, n = 4, 20000
    rng = np.random.default_rng(602)
    E = rng.uniform(0, 1, res ** 3).astype(np.float32)
    E[rng.choice(res ** 3, 6, replace=False)] = 0.0
    E[3] = 1e-6  # below max / 65535: no points
    pts = oracle.adaptive_points(oracle.adaptive_cdf(E, res), seed=11, step=4, n=n)
    cnt = np.bincount(_voxel_of(pts, res), minlength=res ** 3)
    Ed = E.astype(np.float64)
    e = 65535.0 * Ed / Ed.max()
    Qlo = e.sum() - 1.004 * res ** 3
    exact = n * Ed / Ed.sum()
    bound = 1 + n * (1 + res ** 3 * e / e.sum()) * 1.004 / Qlo
    assert np.all(np.abs(cnt - exact) <= bound), np.max(np.abs(cnt - exact) - bound)
    assert cnt.sum() == n and cnt[3] == 0 and np.all(cnt[E == 0] == 0)


# ---------------------------------------------------------------- tolerance bounds
def test_error_bounds_of_a_linear_layer():
    """One linear layer rho = W v + b: with only the input term of the
    precision model (|dv_j| <= in_abs, <= in_rel |v_j|, or for the latent
    inputs <= lat_w sum_k w_k |G_k|) the bound is lambda sqrt(sum_j (W_j
    dv_j)^2), lambda = 6 (Hoeffding at 3e-8); the bounds are linear in the
    precision model."""
    p = synth.random_params(R=4, F=4, m=3, layers=1, width=8, act=synth.ACT_SINE, seed=611)
    on = oracle.OracleNet(p)
    pts = np.random.default_rng(612).uniform(0, 1, (5, 3))
    W = np.asarray(p["weights"][0], np.float64)[0]
    d = 1e-4
    B, _ = oracle.error_bounds(on, pts, (0, d, 0, 0, 0, 0, 0, 0, 0, 0), grad=False)
    np.testing.assert_allclose(B[:, 0], 6 * d * np.linalg.norm(W), rtol=1e-12)
    # in_rel: the input vector [p, sin(Fp), cos(Fp), z] from the oracle's own Fourier matrix and latent grid
    B2, _ = oracle.error_bounds(on, pts, (d, 0, 0, 0, 0, 0, 0, 0, 0, 0), grad=False)
    F = np.asarray(p["fourier"], np.float64)
    for k, x in enumerate(pts):
        e = F @ x
        z = oracle.trilinear(np.asarray(p["grid"], np.float64)[0], x)
        v = np.concatenate([x, np.sin(e), np.cos(e), z])
        assert abs(B2[k, 0] - 6 * d * np.linalg.norm(W * v)) < 1e-12
    # lat_w: the FP16-rounded trilinear weights, 2^-11 of sum_k w_k |G_kc| per latent input
    B3, _ = oracle.error_bounds(on, pts, (0, 0, 0, 0, 0, 0, 0, 0, 0, d), grad=False)
    for k, x in enumerate(pts):
        za = oracle.trilinear(np.abs(np.asarray(p["grid"], np.float64)[0]), x)
        assert abs(B3[k, 0] - 6 * d * np.linalg.norm(W[3 + 2 * 3:] * za)) < 1e-12
    q = synth.random_params(R=4, F=4, m=3, layers=3, width=8, act=synth.ACT_SNAKEALT, seed=613)
    oq = oracle.OracleNet(q)
    prec = np.array(oracle.PREC_FP16)
    Bo1, Bg1 = oracle.error_bounds(oq, pts, prec)
    Bo2, Bg2 = oracle.error_bounds(oq, pts, 2 * prec)
    np.testing.assert_allclose(Bo2, 2 * Bo1, rtol=1e-9)
    np.testing.assert_allclose(Bg2, 2 * Bg1, rtol=1e-6)
