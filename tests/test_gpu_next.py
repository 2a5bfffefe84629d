"""GPU parity of the widened rows: the direct time encoding (Section 7) in
the FP32 and FP16 paths and in the fit."""
import numpy as np
import pytest

import oracle
from paper_2112_01579_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srn():
    import torch
    from paper_2112_01579_gb300 import build
    build.build()
    from paper_2112_01579_gb300 import srn as S
    assert torch.cuda.is_available()
    return S


def _time_params(seed, R=16):
    return synth.random_params(R=R, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=seed,
                               grid_std=0.5, bias_std=0.2, n_keyframes=5, key_times=[0, 4, 8, 12, 15],
                               time_input=1)


@pytest.mark.parametrize("precision", [0, 1])
def test_direct_time_render_and_eval(srn, precision):
    """The time value as one more input after the latent vector (d_0 = 48,
    filling the padding slot of the paper's 48-channel input)."""
    import torch
    S = srn
    p = _time_params(100)
    q = synth.to_half_exact(p) if precision else p
    net = S.Network(q, precision=precision)
    on = oracle.OracleNet(q)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    times = [0.0, 2.0, 5.5, 15.0]
    out = torch.zeros((4, 2, 24, 32, 4), device="cuda")
    S.srn_render(net.ctx, cams, tf, S.render_desc(32, 24, 1 / 64, 2.0), out, times=times)
    torch.cuda.synchronize()
    ref, _, _ = oracle.render(on, cams, H.oracle_tf(tf), 32, 24, 1 / 64, 2.0, times=times)
    tol = H.TOL_FP16_IMG if precision else H.TOL_FP32_IMG
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"direct time, precision {precision}: max image error {err:.2e}")
    assert err <= tol
    pts = np.random.default_rng(101).uniform(0, 1, (20000, 3)).astype(np.float32)
    for t in [1.0, 9.25]:
        o = torch.zeros((len(pts), 1), device="cuda")
        S.srn_eval(net.ctx, torch.tensor(pts, device="cuda"), o, time=t)
        torch.cuda.synchronize()
        err = H.rel_density_err(o.cpu().numpy(), oracle.net_forward(on, pts, t))
        assert err.max() <= (H.TOL_FP16_RHO if precision else H.TOL_FP32_RHO), err.max()


def test_direct_time_fit_step(srn):
    import torch
    S = srn
    vol = synth.blobs_volume(48, 6, seed=102).numpy()
    p = synth.init_params(R=8, F=16, m=14, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=103, n_keyframes=2,
                          key_times=[0.0, 1.0], time_input=1)
    net = S.Network(p, max_fit_points=4000, adam=True)
    on = oracle.OracleNet(p)
    n_par = on.grid.size + on.W.size + on.b.size
    m, v = np.zeros(n_par), np.zeros(n_par)
    loss = torch.zeros(1, device="cuda")
    for s in range(2):
        S.srn_fit_step(net.ctx, torch.tensor(vol, device="cuda"), 4000, 7, s, loss, time=0.4)
        torch.cuda.synchronize()
        lo, grads, st = oracle.fit_step(on, m, v, vol, 4000, 7, s, 1e-2, 5e-3, t=0.4)
        assert abs(float(loss.item()) - lo) <= 1e-5 * max(lo, 1e-3)
    got = net.unpack()
    Wg = np.concatenate([w.ravel() for w in got["weights"]])
    g = grads[on.grid.size:on.grid.size + on.W.size]
    big = np.abs(g) > 1e-2 * np.abs(g).max()
    assert np.abs(Wg - on.W)[big].max() <= 5e-3 * 5e-3 + 1e-7


def _quantize_np(grid, F):
    return H.quantize_u8(grid, F)


def test_u8_grid_codes_are_exact(srn):
    """Section 4.2 8-bit latent grid: per-channel min / max over all keyframes
    and vertices, codes round((g - lo) / step).  Integer results: bit-exact."""
    import torch
    S = srn
    p = synth.random_params(R=12, F=16, m=14, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=104, n_keyframes=2,
                            key_times=[0.0, 1.0])
    p["grid"][..., 3] = 0.25  # a constant channel: step 1, codes 0
    net = S.Network(synth.to_half_exact(p), precision=S.SRN_PREC_FP16, grid_u8=True)
    torch.cuda.synchronize()
    code, lo, step = _quantize_np(net.grid.cpu().numpy(), 16)
    assert np.array_equal(net.grid_q.cpu().numpy(), code)
    qp = net.grid_qp.cpu().numpy()
    assert np.array_equal(qp[:, 0], lo) and np.array_equal(qp[:, 1], step)
    assert qp[3, 1] == 1.0 and np.all(code.reshape(-1, 16)[:, 3] == 0)


@pytest.mark.parametrize("kind", ["render", "eval"])
def test_u8_grid_parity(srn, kind):
    """The FP16 path on the 8-bit grid against the oracle evaluated on the
    dequantized grid lo + step * code."""
    import torch
    S = srn
    p = synth.to_half_exact(H.cfg2_params(seed=105))
    net = S.Network(p, precision=S.SRN_PREC_FP16, grid_u8=True)
    on = oracle.OracleNet(H.u8_params(p))
    if kind == "render":
        tf = synth.tf_preset(8)
        cams = synth.orbit_cameras(2)
        out = torch.zeros((1, 2, 40, 48, 4), device="cuda")
        S.srn_render(net.ctx, cams, tf, S.render_desc(48, 40, 1 / 128, 0.99), out)
        torch.cuda.synchronize()
        ref, mg, _ = oracle.render(on, cams, H.oracle_tf(tf), 48, 40, 1 / 128, 0.99, want_margin=True)
        r = H.compare_images(out.cpu().numpy(), ref, mg, H.TOL_FP16_IMG, 0.99)
        assert r["ok"], r
    else:
        pts = np.random.default_rng(106).uniform(0, 1, (50000, 3)).astype(np.float32)
        o = torch.zeros((len(pts), 1), device="cuda")
        S.srn_eval(net.ctx, torch.tensor(pts, device="cuda"), o)
        torch.cuda.synchronize()
        err = H.rel_density_err(o.cpu().numpy(), oracle.net_forward(on, pts))
        print(f"8-bit grid eval: max relative density error vs FP64 {err.max():.2e}")
        assert err.max() <= H.TOL_FP16_RHO, err.max()


def test_u8_grid_follows_the_fit(srn):
    import torch
    S = srn
    vol = torch.tensor(synth.blobs_volume(48, 6, seed=107).numpy(), device="cuda")
    p = synth.init_params(R=16, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=108)
    net = S.Network(p, precision=S.SRN_PREC_FP16, max_fit_points=1 << 14, adam=True, grid_u8=True)
    loss = torch.zeros(1, device="cuda")
    for s in range(5):
        S.srn_fit_step(net.ctx, vol, 1 << 14, 3, s, loss)
    torch.cuda.synchronize()
    code, lo, step = _quantize_np(net.grid.cpu().numpy(), 16)
    assert np.array_equal(net.grid_q.cpu().numpy(), code)
