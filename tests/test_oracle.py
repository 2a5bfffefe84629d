"""Pins of the FP64 oracle against facts fixed by the paper and mathematics.

Each test checks the oracle against something other than itself: printed
values (tests/golden), closed forms, library routines (torch float64,
grid_sample, torch.optim.Adam), invariants and brute-force finite differences.
No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2112_01579_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _net(params):
    return oracle.OracleNet(params)


def _const_tf(rgb, a, scale):
    return oracle.OracleTF([0.0, 1.0], [list(rgb) + [a], list(rgb) + [a]], scale)


def _nerf_exact(m):
    """Eq. 1 in float64: row k = 2 pi 2^(k div 3) e_(k mod 3)."""
    F = np.zeros((m, 3))
    for k in range(m):
        F[k, k % 3] = 2 * math.pi * 2 ** (k // 3)
    return F


def test_synth_fourier_matrix_is_eq1_in_float32():
    np.testing.assert_array_equal(synth.nerf_fourier_matrix(14), _nerf_exact(14).astype(np.float32))


def _params_linear(F=2, m=3, R=3, D=1, W=None, b=None, grid=None, act=synth.ACT_SINE):
    """Single linear layer network (l = 1): out = W v0 + b."""
    d0 = 3 + 2 * m + F
    W = np.zeros((D, d0)) if W is None else np.asarray(W, dtype=np.float64).reshape(D, d0)
    b = np.zeros(D) if b is None else np.asarray(b, dtype=np.float64).reshape(D)
    if grid is None:
        grid = np.zeros((1, R, R, R, F))
    return dict(grid=grid, fourier=_nerf_exact(m), weights=[W], biases=[b], act=act, key_times=np.zeros(1))


# ---------------------------------------------------------------- RNG
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_sampler_range_and_uniformity():
    P = oracle.sample_points(seed=1234, step=3, n=20000)
    assert P.min() >= 0.0 and P.max() < 1.0
    assert np.all(P * 2 ** 24 == np.floor(P * 2 ** 24))  # multiples of 2^-24 (exact in FP32)
    # mean and variance of U[0,1): 1/2 and 1/12, 6-sigma bounds
    n = len(P)
    assert np.all(np.abs(P.mean(0) - 0.5) < 6 * math.sqrt(1 / 12 / n))
    assert np.all(np.abs(P.var(0) - 1 / 12) < 6 * math.sqrt(1 / 180 / n))
    Q = oracle.sample_points(seed=1234, step=4, n=100)
    assert not np.allclose(P[:100], Q)


# ---------------------------------------------------------------- trilinear
def test_trilinear_reproduces_affine_fields():
    rng = np.random.default_rng(0)
    nx, ny, nz, C = 5, 4, 7, 3
    a = rng.normal(size=C)
    B = rng.normal(size=(C, 3))
    X, Y, Z = np.meshgrid(np.linspace(0, 1, nx), np.linspace(0, 1, ny), np.linspace(0, 1, nz), indexing="xy")
    zz, yy, xx = np.meshgrid(np.linspace(0, 1, nz), np.linspace(0, 1, ny), np.linspace(0, 1, nx), indexing="ij")
    vol = np.stack([a[c] + B[c, 0] * xx + B[c, 1] * yy + B[c, 2] * zz for c in range(C)], axis=-1)
    for _ in range(50):
        p = rng.uniform(0, 1, 3)
        np.testing.assert_allclose(oracle.trilinear(vol, p), a + B @ p, rtol=0, atol=1e-13)
        np.testing.assert_allclose(oracle.trilinear_grad(vol, p), B, rtol=0, atol=1e-12)
    # corners and the far face return stored values
    assert np.allclose(oracle.trilinear(vol, [1, 1, 1]), vol[-1, -1, -1])
    assert np.allclose(oracle.trilinear(vol, [0, 0, 0]), vol[0, 0, 0])
    # positions outside the domain clamp
    assert np.allclose(oracle.trilinear(vol, [1.5, -2, 0.0]), vol[0, 0, -1])


def test_trilinear_matches_grid_sample():
    """torch grid_sample (trilinear, align_corners=True) is vertex aligned."""
    rng = np.random.default_rng(1)
    vol = rng.normal(size=(6, 5, 4, 2))  # [z, y, x, C]
    pts = rng.uniform(0, 1, (40, 3))
    inp = torch.tensor(vol).permute(3, 0, 1, 2)[None]  # [1, C, D, H, W]
    g = torch.tensor(pts * 2 - 1).view(1, 1, 1, -1, 3)
    ref = torch.nn.functional.grid_sample(inp, g, mode="bilinear", align_corners=True)[0, :, 0, 0, :].T.numpy()
    got = np.stack([oracle.trilinear(vol, p) for p in pts])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- network
def test_fourier_and_input_order_by_selectors():
    """Eq. 1 / Eq. 2: v0 = [p, sin(F p), cos(F p), z]; row k of F_NeRF is
    2 pi 2^(k div 3) along axis k mod 3.  A linear net selecting input j
    returns that feature.  The latent grid is affine, so z is known exactly."""
    F, m, R = 2, 7, 4
    d0 = 3 + 2 * m + F
    zz, yy, xx = np.meshgrid(*(np.linspace(0, 1, R),) * 3, indexing="ij")
    grid = np.stack([0.3 + 0.2 * xx - 0.5 * zz, -0.1 + 0.7 * yy], axis=-1)[None]
    rng = np.random.default_rng(2)
    pts = rng.uniform(0, 1, (16, 3))
    for j in range(d0):
        W = np.zeros((1, d0))
        W[0, j] = 1.0
        net = _net(_params_linear(F=F, m=m, R=R, W=W, b=[0.25], grid=grid))
        out = oracle.net_forward(net, pts)[:, 0]
        if j < 3:
            exp = pts[:, j]
        elif j < 3 + m:
            k = j - 3
            exp = np.sin(2 * math.pi * 2 ** (k // 3) * pts[:, k % 3])
        elif j < 3 + 2 * m:
            k = j - 3 - m
            exp = np.cos(2 * math.pi * 2 ** (k // 3) * pts[:, k % 3])
        elif j == 3 + 2 * m:
            exp = 0.3 + 0.2 * pts[:, 0] - 0.5 * pts[:, 2]
        else:
            exp = -0.1 + 0.7 * pts[:, 1]
        np.testing.assert_allclose(out, exp + 0.25, rtol=0, atol=1e-12, err_msg=f"input {j}")


@pytest.mark.parametrize("act,x,expected", [
    (synth.ACT_SINE, math.pi / 2, 1.0),
    (synth.ACT_SINE, math.pi / 6, 0.5),
    (synth.ACT_SNAKEALT, math.pi / 2, math.pi / 4 + 1.0),   # Eq. 3 at pi/2: 0.5 x + 1
    (synth.ACT_SNAKEALT, -math.pi / 2, -math.pi / 4 + 1.0),
    (synth.ACT_SNAKEALT, math.pi / 4, math.pi / 8 + 0.5),
    (synth.ACT_SNAKEALT, math.pi, math.pi / 2),
    (synth.ACT_SNAKEALT, 0.0, 0.0),
])
def test_activation_special_values(act, x, expected):
    """Two-layer selector: hidden_0 = a(x) (bias carries x), out = hidden_0."""
    F, m, c = 1, 1, 3
    d0 = 3 + 2 * m + F
    W0 = np.zeros((c, d0))
    b0 = np.array([x, 0.0, 0.0])
    W1 = np.zeros((1, c))
    W1[0, 0] = 1.0
    p = dict(grid=np.zeros((1, 2, 2, 2, F)), fourier=synth.nerf_fourier_matrix(m).astype(np.float64),
             weights=[W0, W1], biases=[b0, np.zeros(1)], act=act)
    out = oracle.net_forward(_net(p), [[0.3, 0.6, 0.1]])[0, 0]
    assert abs(out - expected) < 1e-14


def _torch_forward(params, pts, t_act):
    """Independent float64 forward with torch library routines: Eq. 2
    features, grid_sample trilinear latent, nn.functional.linear layers."""
    P = torch.tensor(pts)
    Fm = torch.tensor(params["fourier"], dtype=torch.float64)
    e = P @ Fm.T
    g = torch.tensor(params["grid"][0]).permute(3, 0, 1, 2)[None]
    z = torch.nn.functional.grid_sample(g, (P * 2 - 1).view(1, 1, 1, -1, 3), mode="bilinear",
                                        align_corners=True)[0, :, 0, 0, :].T
    v = torch.cat([P, torch.sin(e), torch.cos(e), z], dim=1)
    Ws, bs = params["weights"], params["biases"]
    for i, (W, b) in enumerate(zip(Ws, bs)):
        v = torch.nn.functional.linear(v, torch.tensor(W, dtype=torch.float64), torch.tensor(b, dtype=torch.float64))
        if i < len(Ws) - 1:
            v = t_act(v)
    return v


def test_forward_matches_torch_library_composition():
    p = synth.random_params(R=5, F=4, m=6, layers=4, width=16, out_dim=2, act=synth.ACT_SINE, seed=3)
    p = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    pts = np.random.default_rng(4).uniform(0, 1, (64, 3))
    ref = _torch_forward(p, pts, torch.sin).numpy()
    np.testing.assert_allclose(oracle.net_forward(_net(p), pts), ref, rtol=0, atol=1e-12)


def test_zero_last_layer_gives_constant_field():
    p = synth.random_params(R=4, F=3, m=6, layers=3, width=8, act=synth.ACT_SNAKEALT, seed=5)
    p["weights"][-1] = np.zeros_like(p["weights"][-1])
    p["biases"][-1] = np.array([0.37], np.float32)
    out = oracle.net_forward(_net(p), np.random.default_rng(6).uniform(0, 1, (32, 3)))
    assert np.all(out == np.float32(0.37))


def test_param_gradients_match_finite_differences():
    """Backpropagation vs brute-force central differences in FP64."""
    rng = np.random.default_rng(7)
    p = synth.random_params(R=3, F=2, m=3, layers=3, width=5, out_dim=2, act=synth.ACT_SNAKEALT, seed=8)
    p = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    p["weights"] = [w.astype(np.float64) for w in p["weights"]]
    p["biases"] = [b.astype(np.float64) for b in p["biases"]]
    pts = rng.uniform(0.02, 0.98, (6, 3))
    dout = rng.normal(size=(6, 2))
    net = _net(p)
    dW, db, dg = oracle.net_backward(net, pts, dout)

    def f():
        return float(np.sum(oracle.net_forward(net, pts) * dout))

    h = 1e-6
    for arr, grad in [(net.W, np.concatenate([w.ravel() for w in dW])),
                      (net.b, np.concatenate([b.ravel() for b in db])), (net.grid, dg)]:
        for i in range(arr.size):
            old = arr[i]
            arr[i] = old + h
            fp = f()
            arr[i] = old - h
            fm = f()
            arr[i] = old
            fd = (fp - fm) / (2 * h)
            assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_param_gradients_match_torch_autograd():
    p = synth.random_params(R=4, F=3, m=6, layers=3, width=8, out_dim=1, act=synth.ACT_SINE, seed=9)
    p = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    p["weights"] = [w.astype(np.float64) for w in p["weights"]]
    p["biases"] = [b.astype(np.float64) for b in p["biases"]]
    pts = np.random.default_rng(10).uniform(0, 1, (20, 3))
    dout = np.random.default_rng(11).normal(size=(20, 1))
    Wt = [torch.tensor(w, requires_grad=True) for w in p["weights"]]
    bt = [torch.tensor(b, requires_grad=True) for b in p["biases"]]
    gt = torch.tensor(p["grid"], requires_grad=True)
    P = torch.tensor(pts)
    e = P @ torch.tensor(p["fourier"]).T
    z = torch.nn.functional.grid_sample(gt[0].permute(3, 0, 1, 2)[None], (P * 2 - 1).view(1, 1, 1, -1, 3),
                                        mode="bilinear", align_corners=True)[0, :, 0, 0, :].T
    v = torch.cat([P, torch.sin(e), torch.cos(e), z], dim=1)
    for i in range(3):
        v = torch.nn.functional.linear(v, Wt[i], bt[i])
        if i < 2:
            v = torch.sin(v)
    (v * torch.tensor(dout)).sum().backward()
    dW, db, dg = oracle.net_backward(_net(p), pts, dout)
    for a, b in zip(dW, Wt):
        np.testing.assert_allclose(a, b.grad.numpy(), atol=1e-12)
    for a, b in zip(db, bt):
        np.testing.assert_allclose(a, b.grad.numpy(), atol=1e-12)
    np.testing.assert_allclose(dg.reshape(gt.shape), gt.grad.numpy(), atol=1e-12)


@pytest.mark.parametrize("act", [synth.ACT_SINE, synth.ACT_SNAKEALT])
def test_input_gradient_matches_finite_differences(act):
    p = synth.random_params(R=5, F=4, m=9, layers=4, width=8, act=act, seed=12)
    net = _net(p)
    pts = np.random.default_rng(13).uniform(0.05, 0.95, (10, 3))
    rho, g = oracle.net_input_grad(net, pts)
    np.testing.assert_allclose(rho, oracle.net_forward(net, pts)[:, 0], atol=0)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (oracle.net_forward(net, pts + e)[:, 0] - oracle.net_forward(net, pts - e)[:, 0]) / (2 * h)
        np.testing.assert_allclose(g[:, a], fd, rtol=1e-6, atol=1e-6)


def test_input_vjp_matches_finite_differences():
    """Backward with respect to the positions of sum_d dout_d out_d for a
    four-output network (Section 5 head): brute-force central differences of
    that sum; the density-only seed equals net_input_grad."""
    p = synth.random_params(R=5, F=4, m=9, layers=3, width=8, out_dim=4, act=synth.ACT_SNAKEALT, seed=14)
    net = _net(p)
    rng = np.random.default_rng(15)
    pts = rng.uniform(0.05, 0.95, (10, 3))
    dout = rng.normal(size=(10, 4))
    g = oracle.net_input_vjp(net, pts, dout)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fp = (oracle.net_forward(net, pts + e) * dout).sum(axis=1)
        fm = (oracle.net_forward(net, pts - e) * dout).sum(axis=1)
        np.testing.assert_allclose(g[:, a], (fp - fm) / (2 * h), rtol=1e-6, atol=1e-6)
    e0 = np.zeros((10, 4))
    e0[:, 0] = 1.0
    np.testing.assert_allclose(oracle.net_input_vjp(net, pts, e0), oracle.net_input_grad(net, pts)[1], atol=0)


def test_time_interpolation_is_trilerp_of_lerped_grid():
    """Section 7: the latent vector is interpolated linearly in time between
    keyframes.  By linearity this equals trilinear interpolation of the
    linearly blended grid; at keyframe times it is that keyframe."""
    p = synth.random_params(R=4, F=3, m=3, layers=2, width=6, act=synth.ACT_SNAKEALT, n_keyframes=3, seed=14,
                            key_times=[0.0, 1.0, 3.0])
    net = _net(p)
    pts = np.random.default_rng(15).uniform(0, 1, (12, 3))

    def static(g):
        q = dict(p)
        q["grid"] = g[None]
        q["key_times"] = np.zeros(1)
        return oracle.net_forward(_net(q), pts)

    G = p["grid"].astype(np.float64)
    for t, g in [(2.0, 0.5 * G[1] + 0.5 * G[2]), (0.25, 0.75 * G[0] + 0.25 * G[1]), (1.0, G[1]), (0.0, G[0]),
                 (-1.0, G[0]), (5.0, G[2]), (3.0, G[2])]:
        np.testing.assert_allclose(oracle.net_forward(net, pts, t), static(g), atol=1e-12, err_msg=str(t))


# ---------------------------------------------------------------- TF / camera / box
def test_transfer_function_piecewise_linear():
    tf = oracle.OracleTF([0.2, 0.5, 0.5, 0.9], [[0, 0, 0, 0], [1, 0.5, 0, 0.4], [0, 1, 0, 0.8], [0, 0, 1, 1]], 7.0)
    np.testing.assert_allclose(oracle.tf_eval(tf, -3.0), [0, 0, 0, 0])
    np.testing.assert_allclose(oracle.tf_eval(tf, 0.2), [0, 0, 0, 0])
    np.testing.assert_allclose(oracle.tf_eval(tf, 0.35), [0.5, 0.25, 0, 0.2], atol=1e-15)
    np.testing.assert_allclose(oracle.tf_eval(tf, 0.5), [0, 1, 0, 0.8])  # duplicate point: right segment
    np.testing.assert_allclose(oracle.tf_eval(tf, 0.6), [0, 0.75, 0.25, 0.85], atol=1e-15)
    np.testing.assert_allclose(oracle.tf_eval(tf, 1.7), [0, 0, 1, 1])


def test_camera_center_ray_and_field_of_view():
    # the C ABI takes FP32 cameras: the closed forms use the same FP32 values
    r32 = lambda v: [float(np.float32(x)) for x in v]
    cam = dict(eye=r32([0.3, -1.2, 2.0]), target=r32([0.1, 0.2, -0.3]), up=[0, 1, 0],
               fovy=float(np.float32(math.radians(60))))
    half = 0.5 * cam["fovy"]
    W, H = 9, 7
    o, d = oracle.camera_ray(cam, W, H, 4, 3)
    f = np.subtract(cam["target"], cam["eye"])
    np.testing.assert_allclose(d, f / np.linalg.norm(f), atol=1e-15)
    np.testing.assert_allclose(o, cam["eye"])
    # top-centre pixel: angle to the axis is atan((1 - 1/H) tan(fovy/2)), and it tilts up
    _, d0 = oracle.camera_ray(cam, W, H, 4, 0)
    ang = math.acos(np.clip(np.dot(d0, f / np.linalg.norm(f)), -1, 1))
    assert abs(ang - math.atan((1 - 1 / H) * math.tan(half))) < 1e-12
    assert d0[1] > d[1]
    # left-middle pixel: horizontal half-angle uses the aspect ratio
    _, d1 = oracle.camera_ray(cam, W, H, 0, 3)
    ang = math.acos(np.clip(np.dot(d1, f / np.linalg.norm(f)), -1, 1))
    assert abs(ang - math.atan((1 - 1 / W) * math.tan(half) * W / H)) < 1e-12


def test_box_intersection():
    hit, t0, t1 = oracle.box_intersect([0, 0, 2], [0, 0, -1])
    assert hit and abs(t0 - 1.5) < 1e-15 and abs(t1 - 2.5) < 1e-15
    hit, t0, t1 = oracle.box_intersect([0.1, 0.2, 0.0], [1, 0, 0])
    assert hit and t0 == 0.0 and abs(t1 - 0.4) < 1e-15
    hit, _, _ = oracle.box_intersect([0.7, 0, 2], [0, 0, -1])
    assert not hit
    hit, _, _ = oracle.box_intersect([0, 0, 2], [0, 0, 1])
    assert not hit
    s = 1 / math.sqrt(3)
    hit, t0, t1 = oracle.box_intersect([1, 1, 1], [-s, -s, -s])
    assert hit and abs((t1 - t0) - math.sqrt(3)) < 1e-14


# ---------------------------------------------------------------- render closed forms
def _axis_cam(eye):
    up = [0, 1, 0] if abs(eye[1]) < 1e-9 else [1, 0, 0]
    return dict(eye=eye, target=[0, 0, 0], up=up, fovy=math.radians(40))


@pytest.mark.parametrize("eye,L", [([0, 0, 2.5], 1.0), ([0, 3.0, 0], 1.0),
                                   ([1.5, 1.5, 1.5], math.sqrt(3))])
@pytest.mark.parametrize("ds", [0.03, 1 / 64])
def test_constant_slab_transmittance(eye, L, ds):
    """Constant density: prod_k exp(-kappa l_k) = exp(-kappa L) exactly,
    premultiplied colour = c (1 - exp(-kappa L))."""
    rho0, rgb, a, scale = 0.6, [0.2, 0.7, 0.4], 0.5, 3.0
    ds = float(np.float32(ds))  # the C ABI's FP32 step, as the oracle receives it
    rgb = [float(np.float32(c)) for c in rgb]
    net = _net(_params_linear(b=[rho0]))
    tf = _const_tf(rgb, a, scale)
    W = H = 5
    img, _, ns = oracle.render(net, [_axis_cam(eye)], tf, W, H, ds, et=2.0)
    A = 1 - math.exp(-a * scale * L)
    np.testing.assert_allclose(img[0, 0, 2, 2], [rgb[0] * A, rgb[1] * A, rgb[2] * A, A], atol=1e-14)
    n_expected = math.ceil(L / ds - 1e-12)
    px, _, ns1 = oracle.render(net, [_axis_cam(eye)], tf, W, H, ds, 2.0, pixels=[2 * W + 2])
    assert ns1 == n_expected


def test_early_termination_step_index():
    """Termination after the first sample with A >= et: with full segments
    A_k = 1 - exp(-kappa k ds), so k* = ceil(ln(1/(1-et)) / (kappa ds))."""
    # the C ABI's FP32 step and threshold, as the oracle receives them
    kappa_a, scale, ds, et = 1.0, 37.0, float(np.float32(1 / 100)), float(np.float32(0.99))
    net = _net(_params_linear(b=[0.5]))
    tf = _const_tf([1, 1, 1], kappa_a, scale)
    out, mg, ns = oracle.render(net, [_axis_cam([0, 0, 2.5])], tf, 3, 3, ds, et, pixels=[4], want_margin=True)
    k = math.ceil(math.log(1 / (1 - et)) / (scale * ds))
    assert ns == k
    assert abs(out[0, 3] - (1 - math.exp(-scale * ds * k))) < 1e-14
    assert mg[0] > 1e-4  # this setup is far from a termination tie


def test_miss_and_background():
    net = _net(_params_linear(b=[1.0]))
    tf = _const_tf([1, 1, 1], 1.0, 5.0)
    cam = dict(eye=[0, 0, 3], target=[0, 0, 6], up=[0, 1, 0], fovy=math.radians(30))
    img, _, ns = oracle.render(net, [cam], tf, 4, 4, 0.01, 0.99)
    assert ns == 0 and np.all(img == 0)


@pytest.mark.parametrize("shading", [oracle.SHADE_ADJOINT, oracle.SHADE_FD, oracle.SHADE_HEAD])
def test_shaded_linear_ramp(shading):
    """rho = g p_x + r0 has gradient (g, 0, 0).  Headlight Blinn-Phong: along
    -x, |n.L| = 1 and rgb' = 0.7 rgb + 0.3; along -z, |n.L| = 0 and rgb' =
    0.1 rgb.  The TF ignores density (constant), so A = 1 - exp(-kappa)."""
    g, r0 = 0.2, 0.4
    m, F = 3, 2
    d0 = 3 + 2 * m + F
    D = 4 if shading == oracle.SHADE_HEAD else 1
    W = np.zeros((D, d0))
    W[0, 0] = g
    b = np.zeros(D)
    b[0] = r0
    if D == 4:
        b[1] = g  # head predicts the gradient directly
    net = _net(_params_linear(F=F, m=m, D=D, W=W, b=b))
    rgb, a, scale = np.array([0.5, 0.2, 0.9]), 0.8, 2.0
    tf = _const_tf(rgb, a, scale)
    A = 1 - math.exp(-a * scale)
    for eye, rgb_s in [([2.5, 0, 0], 0.7 * rgb + 0.3), ([0, 0, 2.5], 0.1 * rgb)]:
        out, _, _ = oracle.render(net, [_axis_cam(eye)], tf, 3, 3, 1 / 50, 2.0, shading=shading, fd_h=1 / 64,
                                  pixels=[4])
        np.testing.assert_allclose(out[0], list(rgb_s * A) + [A], atol=1e-12)


def test_dense_dvr_gaussian_blob_matches_erf():
    """Isotropic Gaussian rho = exp(-|x|^2 / (2 s^2)) centred in the box, a
    linear ramp TF (kappa = scale * rho), centre ray along -z:
    A = 1 - exp(-scale * s sqrt(2 pi) erf(0.5 / (s sqrt 2))).  Error bound:
    the linear-interpolation error h^2/8 max|rho''| over the unit chord plus
    the midpoint-rule error ds^2/24 max|rho''|."""
    n, s, scale = 129, 0.1, 4.0
    x = np.linspace(-0.5, 0.5, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    vol = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * s * s))
    tf = oracle.OracleTF([0.0, 1.0], [[1, 1, 1, 0], [1, 1, 1, 1]], scale)
    ds = 1 / 1024
    out, _, _ = oracle.dvr_dense(vol, [_axis_cam([0, 0, 2.5])], tf, 3, 3, ds, 2.0, pixels=[4])
    integral = s * math.sqrt(2 * math.pi) * math.erf(0.5 / (s * math.sqrt(2)))
    exact = 1 - math.exp(-scale * integral)
    h = 1 / (n - 1)
    bound = scale * (h * h / 8 + ds * ds / 24) / (s * s)
    assert abs(out[0, 3] - exact) <= bound
    # an off-centre ray parallel to the axis: the transverse factor is exact
    cam = dict(eye=[0.125, 0.0, 2.5], target=[0.125, 0.0, 0.0], up=[0, 1, 0], fovy=math.radians(40))
    out, _, _ = oracle.dvr_dense(vol, [cam], tf, 3, 3, ds, 2.0, pixels=[4])
    exact = 1 - math.exp(-scale * integral * math.exp(-0.125 ** 2 / (2 * s * s)))
    assert abs(out[0, 3] - exact) <= bound


def test_fv_srn_and_dense_agree_on_identical_fields():
    """A linear net selecting latent channel 0 over a 1-channel latent grid is
    the same field as dense DVR of that grid: images must coincide."""
    R, m, F = 6, 2, 1
    rng = np.random.default_rng(16)
    vol = rng.uniform(0, 1, (R, R, R))
    d0 = 3 + 2 * m + F
    W = np.zeros((1, d0))
    W[0, 3 + 2 * m] = 1.0
    net = _net(_params_linear(F=F, m=m, R=R, W=W, grid=vol[None, ..., None]))
    tf = oracle.OracleTF(*[synth.tf_preset(4)[k] for k in ("pos", "rgba", "opacity_scale")])
    cams = synth.orbit_cameras(2)
    a, _, na = oracle.render(net, cams, tf, 12, 10, 1 / 40, 0.99)
    b, _, nb = oracle.dvr_dense(vol, cams, tf, 12, 10, 1 / 40, 0.99)
    np.testing.assert_allclose(a[0], b, atol=1e-14)
    assert na == nb


# ---------------------------------------------------------------- fit
def test_fit_loss_gradient_matches_finite_differences():
    """Section 5 world-space L1 fit on a 16^3 volume: analytic gradient vs
    central differences of the loss (FP64)."""
    vol = synth.blobs_volume(16, 4, seed=17).numpy()
    p = synth.random_params(R=4, F=2, m=3, layers=2, width=6, act=synth.ACT_SINE, seed=18)
    net = _net(p)
    n, seed, step = 64, 99, 5
    loss, dW, db, dg = oracle.fit_loss_grad(net, vol, n, seed, step)
    grad = np.concatenate([dg, np.concatenate([w.ravel() for w in dW]), np.concatenate([b.ravel() for b in db])])
    arrays = [net.grid, net.W, net.b]
    h = 1e-7
    off = 0
    for arr in arrays:
        for i in range(arr.size):
            old = arr[i]
            arr[i] = old + h
            lp = oracle.fit_loss_grad(net, vol, n, seed, step)[0]
            arr[i] = old - h
            lm = oracle.fit_loss_grad(net, vol, n, seed, step)[0]
            arr[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[off + i]) <= 1e-6 * max(1.0, abs(fd)), (off + i, fd, grad[off + i])
        off += arr.size
    # loss is the mean absolute residual of the drawn points
    pts = oracle.sample_points(seed, step, n)
    y = np.array([oracle.trilinear(vol, q)[0] for q in pts])
    assert abs(loss - np.mean(np.abs(oracle.net_forward(net, pts)[:, 0] - y))) < 1e-14


def test_fit_head_loss_gradient_matches_finite_differences():
    vol = synth.blobs_volume(16, 4, seed=19).numpy()
    p = synth.random_params(R=3, F=2, m=3, layers=2, width=5, out_dim=4, act=synth.ACT_SNAKEALT, seed=20)
    net = _net(p)
    args = (vol, 32, 7, 0, 0.0, 0.5, 0.05)
    loss, dW, db, dg = oracle.fit_loss_grad(net, *args)
    grad = np.concatenate([dg, np.concatenate([w.ravel() for w in dW]), np.concatenate([b.ravel() for b in db])])
    h = 1e-7
    off = 0
    for arr in [net.grid, net.W, net.b]:
        for i in range(arr.size):
            old = arr[i]
            arr[i] = old + h
            lp = oracle.fit_loss_grad(net, *args)[0]
            arr[i] = old - h
            lm = oracle.fit_loss_grad(net, *args)[0]
            arr[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[off + i]) <= 1e-6 * max(1.0, abs(fd))
        off += arr.size


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(21)
    theta = rng.normal(size=5)
    m, v = np.zeros(5), np.zeros(5)
    tp = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    for step in range(6):
        g = rng.normal(size=5) * 10 ** rng.uniform(-3, 1)
        oracle.adam(theta, m, v, g, 0.01, step)
        tp.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(theta, tp.detach().numpy(), rtol=0, atol=1e-15)


def test_fit_step_equals_gradient_then_adam():
    vol = synth.blobs_volume(16, 4, seed=22).numpy()
    p = synth.init_params(R=4, F=2, m=3, layers=2, width=6, act=synth.ACT_SINE, seed=23)
    a, b = _net(p), _net(p)
    n_par = a.grid.size + a.W.size + a.b.size
    m, v = np.zeros(n_par), np.zeros(n_par)
    loss, grads, st = oracle.fit_step(a, m, v, vol, 128, 5, 0, 1e-2, 5e-3)
    assert st == 0
    l2, dW, db, dg = oracle.fit_loss_grad(b, vol, 128, 5, 0)
    assert loss == l2
    for arr, g, lr in [(b.grid, dg, 1e-2), (b.W, np.concatenate([w.ravel() for w in dW]), 5e-3),
                       (b.b, np.concatenate([x.ravel() for x in db]), 5e-3)]:
        tp = torch.tensor(arr.copy(), requires_grad=True)
        # the learning rates are FP32 values at the C ABI (and so in the oracle)
        opt = torch.optim.Adam([tp], lr=float(np.float32(lr)), betas=(0.9, 0.999), eps=1e-8)
        tp.grad = torch.tensor(g)
        opt.step()
        arr[:] = tp.detach().numpy()
    np.testing.assert_allclose(a.grid, b.grid, atol=1e-15)
    np.testing.assert_allclose(a.W, b.W, atol=1e-15)
    np.testing.assert_allclose(a.b, b.b, atol=1e-15)


def test_fit_reduces_loss():
    vol = synth.blobs_volume(16, 4, seed=24).numpy()
    p = synth.init_params(R=4, F=4, m=6, layers=2, width=16, act=synth.ACT_SNAKEALT, seed=25)
    net = _net(p)
    n_par = net.grid.size + net.W.size + net.b.size
    m, v = np.zeros(n_par), np.zeros(n_par)
    losses = [oracle.fit_step(net, m, v, vol, 512, 1, s, 1e-2, 5e-3)[0] for s in range(60)]
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5])


def test_fit_nonfinite_leaves_parameters():
    vol = synth.blobs_volume(16, 4, seed=26).numpy()
    vol[3, 4, 5] = np.nan
    vol[:] = np.nan
    p = synth.init_params(R=4, F=2, m=3, layers=2, width=6, seed=27)
    net = _net(p)
    before = net.W.copy()
    n_par = net.grid.size + net.W.size + net.b.size
    loss, _, st = oracle.fit_step(net, np.zeros(n_par), np.zeros(n_par), vol, 16, 1, 0, 1e-2, 5e-3)
    assert st == 1 and not math.isfinite(loss)
    assert np.array_equal(before, net.W)


# ---------------------------------------------------------------- evaluation
def test_paper_model_sizes():
    """Section 4.2: four layers of 32 channels take about 7.3 kB (FP16) and
    the 32^3 x 16 grid 2 MB at 4 bytes; pins 'layers' = linear layers."""
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))
    d = g["default_network"]
    assert (d["width"] - 4) // 2 == d["m"] == g["fourier_count_rule"]["m"]
    def fp16_kB(layers):
        return 2 * sum(i * o + o for i, o in synth.layer_dims(d["F"], d["m"], layers, d["width"], 1)) / 1000

    # of the candidate readings, l = number of linear layers lands on 7.3 kB
    best = min(range(2, 8), key=lambda l: abs(fp16_kB(l) - d["net_kB"]))
    assert best == d["layers"] and abs(fp16_kB(best) - d["net_kB"]) < 0.1
    assert d["R"] ** 3 * d["F"] * 4 == d["grid_MB"] * 2 ** 20
    e = g["equal_memory_density_grid"]
    assert round((e["R"] ** 3 * e["F"]) ** (1 / 3)) == e["M"]


def test_lowpass_preserves_constant_and_affine_fields():
    n, M = 17, 9
    x = np.linspace(0, 1, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    const = np.full((n, n, n), 0.42)
    np.testing.assert_allclose(oracle.lowpass_resample(const, M), 0.42, atol=1e-14)
    aff = 0.1 + 0.3 * X - 0.2 * Y + 0.5 * Z
    out = oracle.lowpass_resample(aff, M)
    xm = np.linspace(0, 1, M)
    Zm, Ym, Xm = np.meshgrid(xm, xm, xm, indexing="ij")
    exp = 0.1 + 0.3 * Xm - 0.2 * Ym + 0.5 * Zm
    inner = (slice(2, -2),) * 3  # away from clamp-to-edge borders
    np.testing.assert_allclose(out[inner], exp[inner], atol=1e-13)


def test_psnr_and_ssim_closed_forms():
    rng = np.random.default_rng(28)
    a = rng.uniform(0, 1, (20, 24, 4))
    assert oracle.psnr(a, a) == math.inf
    b = a.copy()
    b[..., :3] += 0.01
    assert abs(oracle.psnr(a, b) - 40.0) < 1e-9
    assert abs(oracle.ssim(a, a) - 1.0) < 1e-12
    # two constant images: SSIM = (2 mu_a mu_b + C1) / (mu_a^2 + mu_b^2 + C1)
    ca, cb = np.full((16, 16, 4), 0.3), np.full((16, 16, 4), 0.6)
    C1 = 0.01 ** 2
    assert abs(oracle.ssim(ca, cb) - (2 * 0.18 + C1) / (0.09 + 0.36 + C1)) < 1e-12


def test_direct_time_input_is_the_last_input():
    """Section 7 'direct' encoding: the time is one more scalar input after
    the latent vector; a linear net selecting it returns the time."""
    F, m = 2, 3
    d0 = 3 + 2 * m + F + 1
    W = np.zeros((1, d0))
    W[0, d0 - 1] = 1.0
    p = dict(grid=np.zeros((2, 3, 3, 3, F)), fourier=_nerf_exact(m), weights=[W], biases=[np.array([0.5])],
             act=synth.ACT_SINE, key_times=np.array([0.0, 2.0]), time_input=1)
    net = _net(p)
    for t in [0.0, 0.7, 1.9, 3.0]:
        out = oracle.net_forward(net, [[0.2, 0.4, 0.6]], t)[0, 0]
        assert out == float(np.float32(t)) + 0.5  # the time is an FP32 value at the C ABI
    # the time input changes nothing else: same net without it and a zero time weight agree
    p2 = synth.random_params(R=4, F=4, m=6, layers=3, width=8, seed=90, time_input=1)
    p2["weights"][0][:, -1] = 0.0
    p3 = dict(p2)
    p3["weights"] = [p2["weights"][0][:, :-1]] + p2["weights"][1:]
    p3["time_input"] = 0
    pts = np.random.default_rng(91).uniform(0, 1, (20, 3))
    np.testing.assert_allclose(oracle.net_forward(_net(p2), pts, 0.8), oracle.net_forward(_net(p3), pts, 0.8),
                               atol=1e-13)


def test_direct_time_gradients_match_finite_differences():
    p = synth.random_params(R=3, F=2, m=3, layers=3, width=5, seed=92, n_keyframes=2, key_times=[0.0, 1.0],
                            time_input=1)
    p = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    p["weights"] = [w.astype(np.float64) for w in p["weights"]]
    p["biases"] = [b.astype(np.float64) for b in p["biases"]]
    net = _net(p)
    pts = np.random.default_rng(93).uniform(0.02, 0.98, (5, 3))
    dout = np.random.default_rng(94).normal(size=(5, 1))
    dW, db, dg = oracle.net_backward(net, pts, dout, 0.35)
    g = np.concatenate([w.ravel() for w in dW])
    h = 1e-6
    for i in range(net.W.size):
        old = net.W[i]
        net.W[i] = old + h
        fp = float(np.sum(oracle.net_forward(net, pts, 0.35) * dout))
        net.W[i] = old - h
        fm = float(np.sum(oracle.net_forward(net, pts, 0.35) * dout))
        net.W[i] = old
        assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-6 * max(1.0, abs(g[i]))
