"""GPU parity of Section 6.2 adaptive resampling: the error grid against the
oracle, the error-proportional fit points bit-exact against the oracle's
sampler given the same error values, and fit steps drawn from it."""
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


@pytest.mark.parametrize("width,res,spv,timed", [(32, 12, 8, False), (48, 7, 3, False), (32, 9, 5, True)])
def test_error_grid_matches_oracle(srn, width, res, spv, timed):
    """Error grid against the oracle; the timed case has three keyframes and
    the direct time input, evaluated between keyframes."""
    import torch
    S = srn
    m = synth.fourier_rows_for_width(width)
    kw = dict(n_keyframes=3, key_times=[0.0, 1.0, 3.0], time_input=1) if timed else {}
    p = synth.random_params(R=8, F=16, m=m, layers=3, width=width, act=synth.ACT_SNAKEALT, seed=600 + width,
                            grid_std=0.5, bias_std=0.2, **kw)
    t = 1.75 if timed else 0.0
    vol = synth.blobs_volume(24, 5, seed=601).numpy()
    net = S.Network(p)
    E = torch.full((res ** 3,), -1.0, device="cuda")
    S.srn_error_grid(net.ctx, torch.tensor(vol, device="cuda"), res, spv, 77, E, time=t)
    torch.cuda.synchronize()
    ref = oracle.error_grid(oracle.OracleNet(p), vol, res, spv, 77, t).reshape(-1)
    got = E.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= H.TOL_FP32_RHO * max(1.0, np.abs(ref).max())


def _net_for_points(S):
    p = synth.init_params(R=4, F=4, m=3, layers=2, width=32, seed=602)
    return S.Network(p, max_fit_points=1 << 16, adam=True)


@pytest.mark.parametrize("res,n", [(6, 777), (128, 3001), (203, 2500)])
def test_adaptive_points_bit_exact(srn, res, n):
    """Same FP32 error values on both sides (a synthetic grid with zero
    voxels and a wide dynamic range): every coordinate equal bit for bit.
    res 203 spans 4,100 prefix-sum blocks (several block sums per thread in
    the second scan level)."""
    import torch
    S = srn
    rng = np.random.default_rng(603 + res)
    E = (rng.uniform(0, 1, res ** 3) ** 4).astype(np.float32)
    E[rng.uniform(0, 1, E.size) < 0.3] = 0.0
    net = _net_for_points(S)
    S.srn_fit_set_sampling(net.ctx, torch.tensor(E, device="cuda"), res)
    pts = torch.zeros((n, 3), device="cuda")
    S.srn_fit_points(net.ctx, n, 12345, 9, pts)
    torch.cuda.synchronize()
    ref = oracle.adaptive_points(oracle.adaptive_cdf(E, res), 12345, 9, n)
    assert np.array_equal(pts.cpu().numpy().astype(np.float64), ref)


def test_uniform_points_and_invalid_grids(srn):
    """No grid, a zero grid: the uniform sampler (bit-exact against the
    oracle); a negative or NaN entry is refused and leaves the sampling as
    it was."""
    import torch
    S = srn
    net = _net_for_points(S)
    n = 1000
    uni = oracle.sample_points(5, 3, n)
    pts = torch.zeros((n, 3), device="cuda")
    for E in (None, torch.zeros(8 ** 3, device="cuda")):
        S.srn_fit_set_sampling(net.ctx, E, 8)
        S.srn_fit_points(net.ctx, n, 5, 3, pts)
        torch.cuda.synchronize()
        assert np.array_equal(pts.cpu().numpy().astype(np.float64), uni)
    good = torch.rand(8 ** 3, device="cuda")
    S.srn_fit_set_sampling(net.ctx, good, 8)
    S.srn_fit_points(net.ctx, n, 5, 3, pts)
    before = pts.clone()
    for bad in (-1.0, float("nan"), float("inf")):
        E = good.clone()
        E[17] = bad
        with pytest.raises(S.SrnError) as e:
            S.srn_fit_set_sampling(net.ctx, E, 8)
        assert e.value.status == S.SRN_ERR_INVALID_ARG
        S.srn_fit_points(net.ctx, n, 5, 3, pts)
        assert torch.equal(pts, before)


@pytest.mark.parametrize("layers", [3, 2])
def test_adaptive_fit_steps_match_oracle(srn, layers):
    """Fit steps drawing their points from an error grid, against the
    oracle: the grid is the oracle's (FP64, rounded to FP32) and both sides
    sample from those same FP32 values.  Three layers (the FP32 fit kernels):
    two steps, loss and updated weights; two layers (the tensor-core point
    kernel): one step under the L1 sign rule (test_gpu_fit._tc_fit_step_check)."""
    import torch
    S = srn
    vol = synth.blobs_volume(40, 6, seed=604).numpy()
    p = synth.init_params(R=8, F=16, m=14, layers=layers, width=32, act=synth.ACT_SNAKEALT, seed=605)
    E = oracle.error_grid(oracle.OracleNet(p), vol, 16, 8, 1).reshape(-1).astype(np.float32)
    cdf = oracle.adaptive_cdf(E, 16)
    if layers == 2:
        from tests.test_gpu_fit import _tc_fit_step_check
        _tc_fit_step_check(S, p, vol, 4000, seed=7, cdf=cdf, err=E)
        return
    net = S.Network(p, max_fit_points=4000, adam=True)
    vol_d = torch.tensor(vol, device="cuda")
    S.srn_fit_set_sampling(net.ctx, torch.tensor(E, device="cuda"), 16)
    on = oracle.OracleNet(p)
    n_par = on.grid.size + on.W.size + on.b.size
    m, v = np.zeros(n_par), np.zeros(n_par)
    loss = torch.zeros(1, device="cuda")
    for s in range(2):
        S.srn_fit_step(net.ctx, vol_d, 4000, 7, s, loss)
        torch.cuda.synchronize()
        lo, grads, st = oracle.fit_step(on, m, v, vol, 4000, 7, s, 1e-2, 5e-3, cdf=cdf)
        assert abs(float(loss.item()) - lo) <= 1e-5 * max(lo, 1e-3)
    got = net.unpack()
    Wg = np.concatenate([w.ravel() for w in got["weights"]])
    g = grads[on.grid.size:on.grid.size + on.W.size]
    big = np.abs(g) > 1e-2 * np.abs(g).max()
    assert np.abs(Wg - on.W)[big].max() <= 5e-3 * 5e-3 + 1e-7
