"""Pins of the oracle's Section 6.2 adaptive resampling (error grid and the
error-proportional point distribution) against closed forms and exact counts.
No GPU is needed."""
import numpy as np
import pytest

import oracle
from paper_2112_01579_gb300 import synth


def _const_net(b, R=4, F=4, m=3, layers=3, width=8):
    """A network whose output is the constant b (zero last layer)."""
    p = synth.random_params(R=R, F=F, m=m, layers=layers, width=width, act=synth.ACT_SNAKEALT, seed=501)
    p["weights"][-1] = np.zeros_like(p["weights"][-1])
    p["biases"][-1] = np.array([b], np.float32)
    return oracle.OracleNet(p)


def _axis_ramp(n, axis):
    """Volume [z][y][x] equal to the coordinate along axis (0 = x)."""
    g = np.linspace(0.0, 1.0, n)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    return np.broadcast_to(g.reshape(shape), (n, n, n)).copy()


def test_error_grid_constant_network_constant_volume():
    net = _const_net(0.75)
    E = oracle.error_grid(net, np.full((9, 9, 9), 0.2), 4, 8, seed=3)
    assert E.shape == (4, 4, 4)
    assert np.all(np.abs(E - 0.55) < 1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_error_grid_samples_lie_in_their_voxel(axis):
    """Constant network 2 against the ramp V = p_axis: E_v = 2 - mean(p_axis)
    over the voxel's samples, so it lies in [2 - (v_a + 1) / res,
    2 - v_a / res] for the voxel's index v_a along that axis (a transposed
    axis or a wrong voxel index breaks it); the slab mean is near the
    voxel-centre value."""
    res, spv = 4, 8
    E = oracle.error_grid(_const_net(2.0), _axis_ramp(9, axis), res, spv, seed=11)
    idx = np.indices((res, res, res))  # (z, y, x)
    va = idx[2 - axis]
    assert np.all(E >= 2.0 - (va + 1) / res - 1e-12)
    assert np.all(E <= 2.0 - va / res + 1e-12)
    for k in range(res):
        slab = E[va == k]
        # 128 uniform samples inside a slab of width 1/4: sd of the mean 0.0064
        assert abs(slab.mean() - (2.0 - (k + 0.5) / res)) < 0.03


def test_quantization_levels():
    E = np.zeros(8, np.float32)
    E[:3] = [0.4, 0.2, 0.1]
    S, _ = oracle.adaptive_cdf(E, 2)
    q = np.diff(S.astype(np.int64))
    assert list(q[:3]) == [65535, 32767, 16383] and np.all(q[3:] == 0)
    with pytest.raises(ValueError):
        oracle.adaptive_cdf(np.array([0.1, -1.0] + [0.0] * 6, np.float32), 2)
    with pytest.raises(ValueError):
        oracle.adaptive_cdf(np.array([0.1, np.nan] + [0.0] * 6, np.float32), 2)


def _voxel_of(pts, res):
    v = np.floor(np.asarray(pts) * res).astype(int).clip(0, res - 1)
    return (v[:, 2] * res + v[:, 1]) * res + v[:, 0]


def test_one_hot_error_puts_every_point_in_that_voxel():
    res = 4
    E = np.zeros(res ** 3, np.float32)
    E[37] = 0.3
    pts = oracle.adaptive_points(oracle.adaptive_cdf(E, res), seed=5, step=2, n=500)
    vz, vy, vx = 37 // 16, (37 // 4) % 4, 37 % 4
    lo = np.array([vx, vy, vz]) / res
    assert np.all(pts >= lo) and np.all(pts <= lo + 1.0 / res)


def test_counts_are_proportional_to_the_error():
    res, n = 4, 1000
    # uniform error: every voxel gets n / 64 points, +-1
    cnt = np.bincount(_voxel_of(oracle.adaptive_points(oracle.adaptive_cdf(np.full(64, 0.5, np.float32), res),
                                                       7, 0, n), res), minlength=64)
    assert cnt.min() >= n // 64 and cnt.max() <= n // 64 + 1 and cnt.sum() == n
    # two voxels in the ratio 1 : 3, the rest zero (never sampled)
    E = np.zeros(64, np.float32)
    E[5], E[60] = 0.1, 0.3
    S = oracle.adaptive_cdf(E, res)
    pts = oracle.adaptive_points(S, 7, 0, n)
    cnt = np.bincount(_voxel_of(pts, res), minlength=64)
    q5, q60 = int(S[0][6] - S[0][5]), int(S[0][61] - S[0][60])
    assert abs(cnt[5] - n * q5 / (q5 + q60)) <= 1 and abs(cnt[60] - n * q60 / (q5 + q60)) <= 1
    assert cnt[5] + cnt[60] == n
    # the stratum order walks the voxels in index order
    v = _voxel_of(pts, res)
    assert np.all(np.diff(v) >= 0)


def test_adaptive_fit_loss_uses_the_adaptive_points():
    """Constant network 2 against V = x with all error in one voxel: the loss
    is 2 - mean(x) over points of that voxel, inside its x-range; the
    gradient still matches central differences (FP64)."""
    res = 4
    E = np.zeros(64, np.float32)
    E[22] = 1.0  # vx = 2
    cdf = oracle.adaptive_cdf(E, res)
    net = _const_net(2.0)
    loss = oracle.fit_loss_grad(net, _axis_ramp(9, 0), 200, 9, 1, cdf=cdf)[0]
    assert 2.0 - 3 / 4 <= loss <= 2.0 - 2 / 4
    vol = synth.blobs_volume(12, 3, seed=19).numpy()
    p = synth.random_params(R=3, F=2, m=3, layers=2, width=4, act=synth.ACT_SINE, seed=20)
    net = oracle.OracleNet(p)
    E = np.random.default_rng(21).uniform(0, 1, 64).astype(np.float32)
    cdf = oracle.adaptive_cdf(E, res)
    loss, dW, db, dg = oracle.fit_loss_grad(net, vol, 48, 9, 3, cdf=cdf)
    h = 1e-7
    for arr, g in ((net.W, np.concatenate([w.ravel() for w in dW])), (net.grid, dg)):
        for i in range(0, arr.size, max(1, arr.size // 12)):
            old = arr[i]
            arr[i] = old + h
            lp = oracle.fit_loss_grad(net, vol, 48, 9, 3, cdf=cdf)[0]
            arr[i] = old - h
            lm = oracle.fit_loss_grad(net, vol, 48, 9, 3, cdf=cdf)[0]
            arr[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
