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
    assert np.abs(out.cpu().numpy() - ref).max() <= tol
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
