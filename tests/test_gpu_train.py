"""Training through torch.autograd with the hand-written backward kernels, and
checkpoint / resume of the fused fit."""
import os

import numpy as np
import pytest

import oracle
from paper_2112_01579_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    from paper_2112_01579_gb300 import build
    build.build()
    from paper_2112_01579_gb300 import autograd as A
    from paper_2112_01579_gb300 import srn as S
    assert torch.cuda.is_available()
    return S, A


def _rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def test_autograd_parameter_and_input_gradients(mods):
    import torch
    S, A = mods
    p = H.cfg2_params(seed=70, R=12)
    m = A.SRNModule(p, max_batch=4096)
    rng = np.random.default_rng(71)
    pts_np = rng.uniform(0.02, 0.98, (2000, 3)).astype(np.float32)
    w_np = rng.normal(size=(2000, 1)).astype(np.float32)
    pts = torch.tensor(pts_np, device="cuda", requires_grad=True)
    out = m(pts)
    (out * torch.tensor(w_np, device="cuda")).sum().backward()
    on = oracle.OracleNet(p)
    np.testing.assert_allclose(out.detach().cpu().numpy(), oracle.net_forward(on, pts_np), atol=1e-5)
    rW, rb, rg = oracle.net_backward(on, pts_np, w_np)
    assert _rel(m.grid.grad.cpu().numpy(), rg) <= 2e-5
    assert _rel(m.weights.grad.cpu().numpy(), np.concatenate([w.ravel() for w in rW])) <= 2e-5
    assert _rel(m.biases.grad.cpu().numpy(), np.concatenate(rb)) <= 2e-5
    _, g = oracle.net_input_grad(on, pts_np)
    assert _rel(pts.grad.cpu().numpy(), g * w_np) <= 1e-4


@pytest.mark.parametrize("shape", ["cfg1", "head", "time"])
def test_input_backward_matches_oracle(mods, shape):
    """srn_input_backward: dpts = sum_d dout_d d out_d / d p (FP32) against
    the oracle's backward with respect to the positions, element by element
    at the FP32 gradient bound (1e-4 of max(|g|, 1) per point); for the
    four-output head every output's gradient enters.  Through autograd too."""
    import torch
    S, A = mods
    t = 0.0
    if shape == "cfg1":
        p = H.cfg1_params(seed=74)
    elif shape == "head":
        p = H.cfg2_params(seed=75, R=12, out_dim=4)
    else:
        p = synth.random_params(R=6, F=8, m=12, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=76, grid_std=0.5,
                                n_keyframes=3, key_times=[0.0, 1.0, 4.0])
        t = 2.5
    m = A.SRNModule(p, max_batch=4096)
    net = m.net
    rng = np.random.default_rng(77)
    n = 3001
    pts_np = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    pts_np[:3] = [[0, 0, 0], [1, 1, 1], [0.5, 1, 0]]
    dout_np = rng.normal(size=(n, net.out_dim)).astype(np.float32)
    pts = torch.tensor(pts_np, device="cuda")
    dpts = torch.full((n, 3), float("nan"), device="cuda")
    S.srn_input_backward(net.ctx, pts, torch.tensor(dout_np, device="cuda"), dpts, time=t)
    torch.cuda.synchronize()
    ref = oracle.net_input_vjp(oracle.OracleNet(p), pts_np, dout_np, t)
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1.0)
    err = (np.abs(dpts.cpu().numpy() - ref) / scale).max()
    assert err <= 1e-4, err
    pg = torch.tensor(pts_np, device="cuda", requires_grad=True)
    (m(pg, t) * torch.tensor(dout_np, device="cuda")).sum().backward()
    assert torch.equal(pg.grad, dpts)
    S.srn_input_backward(net.ctx, torch.zeros((0, 3), device="cuda"), torch.zeros((0, net.out_dim), device="cuda"),
                         torch.zeros((0, 3), device="cuda"))


@pytest.mark.parametrize("precision", [0, 1])
def test_torch_optimizer_trains_the_module(mods, precision):
    """A torch.optim.Adam loop on the L1 loss of Section 5 through the
    autograd binding reduces the loss; the FP16 context renders the updated
    weights (its copies are refreshed before each forward)."""
    import torch
    S, A = mods
    vol = synth.blobs_volume(48, 6, seed=72).cuda()
    p = synth.init_params(R=8, F=16, m=14, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=73)
    m = A.SRNModule(p, precision=precision, max_batch=1 << 14)
    opt = torch.optim.Adam([{"params": [m.grid], "lr": 1e-2}, {"params": [m.weights, m.biases], "lr": 5e-3}])
    g = torch.Generator(device="cuda").manual_seed(0)
    tmp = torch.empty(1, device="cuda")
    losses = []
    for step in range(120):
        pts = torch.rand((1 << 14, 3), device="cuda", generator=g)
        target = torch.nn.functional.grid_sample(vol[None, None], (pts * 2 - 1).view(1, 1, 1, -1, 3),
                                                 align_corners=True).view(-1, 1)
        loss = (m(pts) - target).abs().mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10])


def test_checkpoint_resume_is_bit_exact(mods, tmp_path):
    import torch
    S, A = mods
    vol = torch.tensor(synth.blobs_volume(48, 6, seed=74).numpy(), device="cuda")
    p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=75)
    n = 1 << 14
    loss = torch.zeros(1, device="cuda")
    a = S.Network(p, max_fit_points=n, adam=True)
    for s in range(20):
        S.srn_fit_step(a.ctx, vol, n, 3, s, loss)
        if s == 9:
            path = os.path.join(tmp_path, "ckpt.srn")
            S.srn_save(a.ctx, path, s + 1)
    b = S.Network(p, max_fit_points=n, adam=True)
    start = S.srn_load(b.ctx, path)
    assert start == 10
    for s in range(start, 20):
        S.srn_fit_step(b.ctx, vol, n, 3, s, loss)
    torch.cuda.synchronize()
    assert torch.equal(a.grid, b.grid) and torch.equal(a.weights, b.weights) and torch.equal(a.biases, b.biases)
    assert torch.equal(a.adam_m, b.adam_m) and torch.equal(a.adam_v, b.adam_v)
    # the FP16 copies follow the loaded masters
    assert torch.equal(b.grid_h, b.grid.half())
    # a checkpoint of another shape is refused
    c = S.Network(synth.init_params(R=6, F=8, m=12, layers=2, width=32, seed=76), adam=True)
    with pytest.raises(S.SrnError) as e:
        S.srn_load(c.ctx, path)
    assert e.value.status == S.SRN_ERR_INVALID_ARG
    with pytest.raises(S.SrnError):
        S.srn_load(c.ctx, os.path.join(tmp_path, "missing.srn"))
