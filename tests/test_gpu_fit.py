"""GPU parity of the fit path (sampler, L1 loss, backward through the
network, atomic-free latent-grid gradient, Adam) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2112_01579_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

# FP32 gradients accumulated over thousands of points: error relative to the
# largest entry of each gradient block.
TOL_GRAD = 2e-5
# Gradients of the tensor-core fit (two-layer width-32 density networks):
# every product of v0 / delta with weights or with each other is formed from
# FP16 hi + lo splits, whose residual is <= 2^-22 of each factor, so a term
# carries ~2^-21 of relative error instead of FP32's 2^-24; the sums of
# sign-weighted terms cancel strongly (the L1 gradient), and relative to the
# block maximum the error reaches ~1e-4 (measured 3.5e-5 weights, 8.5e-5
# latent grid).  Still 5x inside the FP16 tensor-core density bound (1e-3).
TOL_GRAD_MMA = 2e-4


def _mma_fit(p):
    """True when the fit step of this network runs the tensor-core point
    kernel (width 32, two layers, density output, no time input)."""
    W = p["weights"]
    m, F = p["fourier"].shape[0], p["grid"].shape[-1]
    return (len(W) == 2 and W[0].shape[0] == 32 and W[1].shape[0] == 1 and not p.get("time_input", 0)
            and (m, F) in ((12, 8), (14, 16)))


@pytest.fixture(scope="module")
def srn():
    import torch
    from paper_2112_01579_gb300 import build
    build.build()
    from paper_2112_01579_gb300 import srn as S
    assert torch.cuda.is_available()
    return S


def _rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("shape", ["cfg1", "cfg2", "head", "time", "dense_cells", "large_9bit", "large_8bit"])
def test_backward_matches_oracle(srn, shape):
    import torch
    S = srn
    t = 0.0
    n = 3001  # ragged against the 128-point CTAs and the 2048-key sort blocks
    if shape in ("large_9bit", "large_8bit"):
        # 100,003 points: the histogram scan runs in several blocks; 7^3 cells
        # sort in one 9-bit pass, 15^3 cells in two 8-bit passes
        p = H.cfg1_params(seed=37) if shape == "large_9bit" else H.cfg2_params(seed=38, R=16)
        n = 100003
    elif shape == "dense_cells":
        # >= 32 points per cell: the (cell, corner)-parallel latent-gradient pass
        p = synth.random_params(R=6, F=16, m=14, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=36,
                                grid_std=0.5, n_keyframes=2, key_times=[0.0, 1.0])
        n, t = 20011, 0.3
    elif shape == "cfg1":
        p = H.cfg1_params(seed=30)
    elif shape == "cfg2":
        p = H.cfg2_params(seed=31, R=16)
    elif shape == "head":
        p = H.cfg2_params(seed=32, R=12, out_dim=4)
    else:
        p = synth.random_params(R=6, F=8, m=12, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=33, grid_std=0.5,
                                n_keyframes=3, key_times=[0.0, 1.0, 4.0])
        t = 2.5
    net = S.Network(p, max_fit_points=n)
    rng = np.random.default_rng(34)
    pts = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    pts[:3] = [[0, 0, 0], [1, 1, 1], [0.5, 1, 0]]
    D = net.out_dim
    dout = rng.normal(size=(n, D)).astype(np.float32)
    dg = torch.empty(net.grid.numel(), device="cuda")
    dW = torch.empty(net.weights.numel(), device="cuda")
    db = torch.empty(net.biases.numel(), device="cuda")
    S.srn_backward(net.ctx, torch.tensor(pts, device="cuda"), torch.tensor(dout, device="cuda"), dg, dW, db, time=t)
    torch.cuda.synchronize()
    rW, rb, rg = oracle.net_backward(oracle.OracleNet(p), pts, dout, t)
    assert _rel(dW.cpu().numpy(), np.concatenate([w.ravel() for w in rW])) <= TOL_GRAD
    assert _rel(db.cpu().numpy(), np.concatenate(rb)) <= TOL_GRAD
    assert _rel(dg.cpu().numpy(), rg) <= TOL_GRAD
    # deterministic: a second call gives bit-identical gradients
    dg2, dW2, db2 = torch.empty_like(dg), torch.empty_like(dW), torch.empty_like(db)
    S.srn_backward(net.ctx, torch.tensor(pts, device="cuda"), torch.tensor(dout, device="cuda"), dg2, dW2, db2,
                   time=t)
    torch.cuda.synchronize()
    assert torch.equal(dg, dg2) and torch.equal(dW, dW2) and torch.equal(db, db2)


def test_backward_empty_and_single_point(srn):
    import torch
    S = srn
    p = H.cfg1_params(seed=35)
    net = S.Network(p, max_fit_points=16)
    dg = torch.full((net.grid.numel(),), 7.0, device="cuda")
    dW = torch.full((net.weights.numel(),), 7.0, device="cuda")
    db = torch.full((net.biases.numel(),), 7.0, device="cuda")
    S.srn_backward(net.ctx, torch.zeros((0, 3), device="cuda"), torch.zeros((0, 1), device="cuda"), dg, dW, db)
    torch.cuda.synchronize()
    assert float(dg.abs().max()) == 0 and float(dW.abs().max()) == 0 and float(db.abs().max()) == 0
    pts = np.array([[0.3, 0.7, 0.2]], np.float32)
    S.srn_backward(net.ctx, torch.tensor(pts, device="cuda"), torch.ones((1, 1), device="cuda"), dg, dW, db)
    torch.cuda.synchronize()
    rW, rb, rg = oracle.net_backward(oracle.OracleNet(p), pts, np.ones((1, 1)))
    assert _rel(dg.cpu().numpy(), rg) <= TOL_GRAD
    with pytest.raises(S.SrnError):
        S.srn_backward(net.ctx, torch.zeros((17, 3), device="cuda"), torch.zeros((17, 1), device="cuda"), dg, dW, db)


def _fit_pair(S, p, vol, n, steps, lr_grid=1e-2, lr_net=5e-3, seed=3, gw=0.0, gs=1.0, t=0.0):
    import torch
    net = S.Network(p, max_fit_points=n, adam=True)
    on = oracle.OracleNet(p)
    n_par = on.grid.size + on.W.size + on.b.size
    m, v = np.zeros(n_par), np.zeros(n_par)
    loss = torch.zeros(1, device="cuda")
    vt = torch.tensor(vol, device="cuda")
    losses = []
    for s in range(steps):
        S.srn_fit_step(net.ctx, vt, n, seed, s, loss, lr_grid=lr_grid, lr_net=lr_net, grad_weight=gw, grad_scale=gs,
                       time=t)
        torch.cuda.synchronize()
        lo, grads, st = oracle.fit_step(on, m, v, vol, n, seed, s, lr_grid, lr_net, t=t, gw=gw, gs=gs)
        losses.append((float(loss.item()), lo))
    return net, on, losses, grads


def _check_params(net, on, grads, lr_grid, lr_net, eps_g=TOL_GRAD):
    """After Adam, entries whose oracle gradient is not tiny must agree
    closely; entries with |g| near zero may differ by up to 2 lr.  Adam
    divides each entry by its own gradient magnitude, so an entry whose
    gradient is a fraction q of the block maximum carries the gradient error
    eps_g / q into its update: with the FP32 bound (eps_g = TOL_GRAD) and
    q >= 1e-2 that is <= 2e-3 lr per step, and over the two steps compared
    here the bound is 5e-3 lr; it scales with eps_g."""
    got = net.unpack()
    ng, nW = on.grid.size, on.W.size
    for arr_gpu, arr_orc, g, lr in [(got["grid"].ravel(), on.grid, grads[:ng], lr_grid),
                                    (np.concatenate([w.ravel() for w in got["weights"]]), on.W, grads[ng:ng + nW],
                                     lr_net),
                                    (np.concatenate(got["biases"]), on.b, grads[ng + nW:], lr_net)]:
        big = np.abs(g) > 1e-2 * np.abs(g).max()
        d = np.abs(arr_gpu.astype(np.float64) - arr_orc)
        assert d[big].max() <= 5e-3 * (eps_g / TOL_GRAD) * lr + 1e-7, d[big].max()
        assert d.max() <= 2 * lr + 1e-6


def _tc_fit_step_check(S, p, vol, n, seed=3, lr_grid=1e-2, lr_net=5e-3, t=0.0, cdf=None, err=None):
    """One tensor-core fit step on targets in [0, 1] against the oracle.  The
    step's gradient (read back as Adam's first moment, m = (1 - beta1) g) must
    pass the L1 sign-validity check; Adam's first update is lr g / (|g| +
    eps), so every parameter whose oracle gradient exceeds its uncertainty
    (the gradient bound plus the undecided points' possible contributions)
    moves exactly as the oracle's, and the others by at most 2 lr.  Only one
    step is compared: where a gradient's sign is undecided the two sides'
    parameters legitimately part by 2 lr, and the next step's residuals and
    signs follow different parameters (multi-step agreement of the step
    pipeline is covered by the FP32 fit and the bit-identical graph replay)."""
    import torch
    net = S.Network(p, max_fit_points=n, adam=True)
    if err is not None:
        S.srn_fit_set_sampling(net.ctx, torch.tensor(err, device="cuda"), round(err.size ** (1 / 3)))
    on = oracle.OracleNet(p)
    n_par = on.grid.size + on.W.size + on.b.size
    m, v = np.zeros(n_par), np.zeros(n_par)
    loss = torch.zeros(1, device="cuda")
    S.srn_fit_step(net.ctx, torch.tensor(vol, device="cuda"), n, seed, 0, loss, lr_grid=lr_grid, lr_net=lr_net,
                   time=t)
    torch.cuda.synchronize()
    g_gpu = net.adam_m.cpu().numpy().astype(np.float64) / 0.1
    lo_chk, g_orc, unc, n_amb, flips = H.l1_fit_gradient_check(g_gpu, p, vol, n, seed, 0, TOL_GRAD_MMA, t=t, cdf=cdf)
    lo, grads, st = oracle.fit_step(on, m, v, vol, n, seed, 0, lr_grid, lr_net, t=t, cdf=cdf)
    assert st == 0 and abs(lo - lo_chk) < 1e-12
    assert abs(float(loss.item()) - lo) <= 1e-5 * max(abs(lo), 1e-3)
    got = net.unpack()
    ng, nW = on.grid.size, on.W.size
    theta_gpu = np.concatenate([got["grid"].ravel(), np.concatenate([w.ravel() for w in got["weights"]]),
                                np.concatenate(got["biases"])]).astype(np.float64)
    theta_orc = np.concatenate([on.grid, on.W, on.b])
    lr = np.concatenate([np.full(ng, lr_grid), np.full(nW + on.b.size, lr_net)])
    decided = np.abs(g_orc) > unc
    d = np.abs(theta_gpu - theta_orc)
    # a decided entry moves by lr g / (|g| + eps) on both sides: the gradient
    # difference (<= unc) changes that by at most eps unc / (|g| - unc)^2,
    # FP32 arithmetic by ~1e-6 relative, the stored value by half an ulp
    eps = 1e-8
    gap = np.maximum(np.abs(g_orc) - unc, 1e-30)
    allowed = lr * (eps * unc / gap ** 2 + 1e-6) + 2.0 ** -23 * np.maximum(np.abs(theta_orc), 1e-30)
    assert np.all(d[decided] <= allowed[decided]), (d[decided] / allowed[decided]).max()
    assert np.all(d <= 2 * lr + 1e-6)
    return n_amb, flips


@pytest.mark.parametrize("shape", ["cfg1", "cfg2"])
def test_fit_step_matches_oracle(srn, shape):
    """Fit steps on a [0, 1] volume.  The four-layer network runs the FP32
    kernels and is compared over two steps; the two-layer network runs the
    tensor-core point kernel and is compared over one step with the L1 sign
    rule (see _tc_fit_step_check)."""
    S = srn
    vol = synth.blobs_volume(64, 8, seed=36).numpy()
    if shape == "cfg1":
        p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=37)
        assert _mma_fit(p)
        _tc_fit_step_check(S, p, vol, 5000)
        return
    p = synth.init_params(R=16, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=38)
    net, on, losses, grads = _fit_pair(S, p, vol, 5000, 2)
    for lg, lo in losses:
        assert abs(lg - lo) <= 1e-5 * max(abs(lo), 1e-3), losses
    _check_params(net, on, grads, 1e-2, 5e-3, TOL_GRAD)


@pytest.mark.parametrize("shape", ["f8_sine", "f16_snake", "f8_gaussian_fourier"])
def test_tensor_core_fit_gradients(srn, shape):
    """The tensor-core fit step's gradient, read back as Adam's first moment
    after one step with zero learning rates (m = (1 - beta1) g), against the
    oracle's loss gradient on a [0, 1] volume: 20,011 points (ragged tiles
    over all warpgroups), both instantiated input shapes, within
    TOL_GRAD_MMA of each block's maximum under the L1 sign rule
    (helpers.l1_fit_gradient_check); the loss within 1e-6.  NeRF Fourier rows
    take the angle-doubling features; a Gaussian Fourier matrix the
    compensated sin/cos of each row."""
    import torch
    S = srn
    vol = synth.blobs_volume(48, 6, seed=42).numpy()
    if shape == "f8_sine":
        p = synth.random_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=43, grid_std=0.3)
    elif shape == "f16_snake":
        p = synth.random_params(R=10, F=16, m=14, layers=2, width=32, act=synth.ACT_SNAKEALT, seed=44, grid_std=0.3)
    else:
        p = synth.random_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=45, grid_std=0.3)
        p["fourier"] = (np.random.default_rng(46).normal(0.0, 6.0, (12, 3))).astype(np.float32)
    assert _mma_fit(p)
    n = 20011
    net = S.Network(p, max_fit_points=n, adam=True)
    loss = torch.zeros(1, device="cuda")
    S.srn_fit_step(net.ctx, torch.tensor(vol, device="cuda"), n, 5, 0, loss, lr_grid=0.0, lr_net=0.0)
    torch.cuda.synchronize()
    g = net.adam_m.cpu().numpy().astype(np.float64) / 0.1
    lo, _, _, n_amb, flips = H.l1_fit_gradient_check(g, p, vol, n, 5, 0, TOL_GRAD_MMA)
    print(f"{shape}: {n_amb} points within the forward bound of r = 0, {flips} took the other sign")
    assert abs(float(loss.item()) - lo) <= 1e-6 * max(abs(lo), 1e-3)


@pytest.mark.parametrize("net_kind", ["init", "random"])
def test_tensor_core_fit_gradients_full_batch(srn, net_kind):
    """The benchmarked fit step: the plain workload's network (8^3 x 8 grid,
    12 Fourier rows, two sine layers of width 32; Xavier initialisation, or
    a random network with a wider grid) on the 256^3 fractal-noise volume
    ([0, 1]) with 2^18 points, gradient and loss against the oracle under
    the L1 sign rule."""
    import torch
    S = srn
    vol_t = synth.noise_volume(256, seed=0, device="cuda").contiguous()
    vol = vol_t.cpu().numpy()
    if net_kind == "init":
        p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=0)
    else:
        p = synth.random_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=47, grid_std=0.3)
    assert _mma_fit(p)
    n = 1 << 18
    net = S.Network(p, max_fit_points=n, adam=True)
    loss = torch.zeros(1, device="cuda")
    S.srn_fit_step(net.ctx, vol_t, n, 1, 0, loss, lr_grid=0.0, lr_net=0.0)
    torch.cuda.synchronize()
    g = net.adam_m.cpu().numpy().astype(np.float64) / 0.1
    lo, _, _, n_amb, flips = H.l1_fit_gradient_check(g, p, vol, n, 1, 0, TOL_GRAD_MMA)
    print(f"{net_kind}: {n_amb} of {n} points within the forward bound of r = 0, {flips} took the other sign")
    assert abs(float(loss.item()) - lo) <= 1e-6 * max(abs(lo), 1e-3)


def test_fit_head_and_keyframes(srn):
    S = srn
    vol = synth.blobs_volume(48, 6, seed=39).numpy()
    p = synth.init_params(R=8, F=16, m=14, layers=3, width=32, out_dim=4, act=synth.ACT_SNAKEALT, seed=40)
    net, on, losses, grads = _fit_pair(S, p, vol, 3000, 2, gw=0.5, gs=0.05)
    for lg, lo in losses:
        assert abs(lg - lo) <= 1e-5 * max(abs(lo), 1e-3), losses
    _check_params(net, on, grads, 1e-2, 5e-3)
    p = synth.init_params(R=6, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=41, n_keyframes=3,
                          key_times=[0.0, 2.0, 3.0])
    assert _mma_fit(p)
    _tc_fit_step_check(S, p, vol, 2000, t=2.25)


def test_fit_is_deterministic_and_reduces_loss(srn):
    import torch
    S = srn
    vol = torch.tensor(synth.blobs_volume(64, 8, seed=42).numpy(), device="cuda")
    p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=43)
    nets = [S.Network(p, max_fit_points=1 << 16, adam=True) for _ in range(2)]
    loss = torch.zeros(1, device="cuda")
    hist = [[], []]
    for k, net in enumerate(nets):
        for s in range(150):
            S.srn_fit_step(net.ctx, vol, 1 << 16, 11, s, loss)
            if s % 10 == 0 or s == 149:
                torch.cuda.synchronize()
                hist[k].append(float(loss.item()))
    assert hist[0] == hist[1]
    assert torch.equal(nets[0].grid, nets[1].grid) and torch.equal(nets[0].weights, nets[1].weights)
    assert hist[0][-1] < 0.5 * hist[0][0]
    st, _ = S.srn_sync_status(nets[0].ctx)
    assert st == 0


def test_fit_nonfinite_leaves_parameters(srn):
    import torch
    S = srn
    vol = synth.blobs_volume(32, 4, seed=44)
    vol[:] = float("nan")
    p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, seed=45)
    net = S.Network(p, max_fit_points=1024, adam=True)
    before = (net.grid.clone(), net.weights.clone(), net.biases.clone())
    loss = torch.zeros(1, device="cuda")
    S.srn_fit_step(net.ctx, vol.cuda(), 1024, 1, 0, loss)
    st, msg = S.srn_sync_status(net.ctx)
    assert st == S.SRN_ERR_NONFINITE, msg
    assert torch.equal(before[0], net.grid) and torch.equal(before[1], net.weights)
    assert torch.equal(before[2], net.biases)
    assert S.srn_sync_status(net.ctx)[0] == 0  # the status word is cleared once read


def test_fit_bounded_wait_reports_timeout(srn, monkeypatch):
    """The fit's timeout path without a fault: with SRN_TEST_STALL=1 the
    tensor-core point kernel issues no MMA, its bounded waits run out, the
    step reports SRN_ERR_TIMEOUT and Adam leaves parameters and moments as
    they were; the next step on the same context equals that step on a fresh
    context bit for bit."""
    import torch
    S = srn
    vol = torch.tensor(synth.blobs_volume(32, 4, seed=46).numpy(), device="cuda")
    p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=47)
    assert _mma_fit(p)
    n = 1 << 14
    net = S.Network(p, max_fit_points=n, adam=True)
    fresh = S.Network(p, max_fit_points=n, adam=True)
    state = lambda m: [t.clone() for t in (m.grid, m.weights, m.biases, m.adam_m, m.adam_v)]
    before = state(net)
    loss = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    monkeypatch.setenv("SRN_TEST_STALL", "1")
    S.srn_fit_step(net.ctx, vol, n, 5, 0, loss)
    torch.cuda.synchronize()
    monkeypatch.delenv("SRN_TEST_STALL")
    st, msg = S.srn_sync_status(net.ctx)
    assert st == S.SRN_ERR_TIMEOUT, (st, msg)
    assert all(torch.equal(a, b) for a, b in zip(before, state(net)))
    loss2 = torch.zeros(1, device="cuda")
    S.srn_fit_step(net.ctx, vol, n, 5, 0, loss)
    S.srn_fit_step(fresh.ctx, vol, n, 5, 0, loss2)
    torch.cuda.synchronize()
    assert S.srn_sync_status(net.ctx)[0] == 0 and S.srn_sync_status(fresh.ctx)[0] == 0
    assert torch.equal(loss, loss2) and bool(torch.isfinite(loss).all())
    assert all(torch.equal(a, b) for a, b in zip(state(net), state(fresh)))
    net.close()
    fresh.close()
