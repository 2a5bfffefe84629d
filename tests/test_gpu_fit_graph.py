"""srn_fit_steps (one fit step captured as a CUDA graph and replayed, the
step index in device memory) against the same number of srn_fit_step calls:
every parameter, Adam moment, FP16 / 8-bit copy and the loss equal bit for
bit.  The single steps are themselves parity-tested against the oracle."""
import pytest

from paper_2112_01579_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srn():
    import torch
    from paper_2112_01579_gb300 import build
    build.build()
    from paper_2112_01579_gb300 import srn as S
    assert torch.cuda.is_available()
    return S


def _params(shape):
    if shape == "tensor_core":  # two-layer width 32: the tensor-core point kernel
        return synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=70), {}
    if shape == "fp32_deep":
        return synth.init_params(R=8, F=16, m=14, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=71), {}
    if shape == "head":
        p = synth.init_params(R=8, F=16, m=14, layers=3, width=32, out_dim=4, act=synth.ACT_SNAKEALT, seed=72)
        return p, dict(grad_weight=0.5, grad_scale=0.05)
    if shape == "grid_u8":  # the 8-bit grid is requantized inside the graph
        p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=73)
        return p, dict(precision=True)
    if shape == "keyframes":
        p = synth.init_params(R=6, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=74, n_keyframes=3,
                              key_times=[0.0, 2.0, 3.0])
        return p, dict(time=2.25)
    raise ValueError(shape)


def _net(S, p, n, fp16):
    if fp16:
        return S.Network(p, precision=S.SRN_PREC_FP16, max_fit_points=n, adam=True, grid_u8=True)
    return S.Network(p, max_fit_points=n, adam=True)


def _state(net):
    out = [net.grid, net.weights, net.biases, net.adam_m, net.adam_v, net.grid_h, net.weights_h]
    if net.grid_q is not None:
        out += [net.grid_q, net.grid_qp]
    return [t.clone() for t in out]


def _same(a, b):
    import torch
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("shape", ["tensor_core", "fp32_deep", "head", "grid_u8", "keyframes"])
def test_fit_steps_equal_single_steps(srn, shape):
    """7 replayed steps from step 0, then 5 more from step 7 (the cached
    graph, the counter restarted), then 3 with other learning rates (a new
    capture): after each run the two networks are identical."""
    import torch
    S = srn
    p, kw = _params(shape)
    fp16 = kw.pop("precision", False)
    vol = torch.tensor(synth.blobs_volume(40, 6, seed=75).numpy(), device="cuda")
    n = 3001
    a, b = _net(S, p, n, fp16), _net(S, p, n, fp16)
    la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    step = 0
    for count, lrs in ((7, (1e-2, 5e-3)), (5, (1e-2, 5e-3)), (3, (2e-2, 1e-3))):
        for s in range(step, step + count):
            S.srn_fit_step(a.ctx, vol, n, 9, s, la, lr_grid=lrs[0], lr_net=lrs[1], **kw)
        S.srn_fit_steps(b.ctx, vol, n, 9, step, count, lb, lr_grid=lrs[0], lr_net=lrs[1], **kw)
        torch.cuda.synchronize()
        step += count
        assert torch.equal(la, lb), (shape, step)
        assert _same(_state(a), _state(b)), (shape, step)
    assert S.srn_sync_status(b.ctx)[0] == 0


def test_fit_steps_with_adaptive_sampling(srn):
    """The adaptive distribution's values are read at replay time: a new
    error grid of the same resolution is used without a new capture."""
    import torch
    S = srn
    vol = torch.tensor(synth.blobs_volume(40, 6, seed=76).numpy(), device="cuda")
    p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=77)
    n = 4000
    a, b = S.Network(p, max_fit_points=n, adam=True), S.Network(p, max_fit_points=n, adam=True)
    la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    E = torch.zeros(16 ** 3, device="cuda")
    step = 0
    for rnd in range(2):
        S.srn_error_grid(a.ctx, vol, 16, 4, rnd, E)
        for net in (a, b):
            S.srn_fit_set_sampling(net.ctx, E, 16)
        for s in range(step, step + 4):
            S.srn_fit_step(a.ctx, vol, n, 3, s, la)
        S.srn_fit_steps(b.ctx, vol, n, 3, step, 4, lb)
        torch.cuda.synchronize()
        step += 4
        assert torch.equal(la, lb) and _same(_state(a), _state(b)), rnd


def test_fit_steps_arguments_and_nonfinite(srn):
    import torch
    S = srn
    p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, seed=78)
    net = S.Network(p, max_fit_points=1024, adam=True)
    vol = torch.tensor(synth.blobs_volume(32, 4, seed=79).numpy(), device="cuda")
    loss = torch.zeros(1, device="cuda")
    before = _state(net)
    S.srn_fit_steps(net.ctx, vol, 1024, 1, 0, 0, loss)  # zero steps: nothing happens
    torch.cuda.synchronize()
    assert _same(before, _state(net))
    for first, count, npts in ((0, -1, 1024), (-1, 2, 1024), (2 ** 31 - 2, 3, 1024), (0, 2, 1025)):
        with pytest.raises(S.SrnError) as e:
            S.srn_fit_steps(net.ctx, vol, npts, 1, first, count, loss)
        assert e.value.status == S.SRN_ERR_INVALID_ARG
    S.srn_fit_steps(net.ctx, vol, 1024, 1, 2 ** 31 - 4, 3, loss)  # first_step + n_steps = INT_MAX
    torch.cuda.synchronize()
    assert S.srn_sync_status(net.ctx)[0] == 0
    bad = vol.clone()
    bad[:] = float("nan")
    before = _state(net)
    S.srn_fit_steps(net.ctx, bad, 1024, 1, 0, 3, loss)
    st, msg = S.srn_sync_status(net.ctx)
    assert st == S.SRN_ERR_NONFINITE, msg
    assert _same(before, _state(net))
