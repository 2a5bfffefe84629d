"""srn_backward_static: the parameter backward for callers that cannot
allocate device memory.

Some integrations may not call cudaMalloc at all: hosts whose device memory
belongs to another allocator (a framework's caching pool or a fixed arena
sized at start-up, where an outside allocation breaks its accounting), and
frame loops that must not take the device-wide synchronization that
cudaMalloc / cudaFree can cause.  srn_backward needs a context (srn_create
allocates its scratch); srn_backward_static takes the network description
directly and works in a fixed device array inside the library.

Its outputs are checked against the FP64 oracle element by element, on two
calls in a row (the second call finds the array as the first one left it),
and against srn_backward as a second check.  The file stands on its own: it
passes alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL_GRAD = 2e-5  # the backward tests' bound: error relative to each block's largest entry


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


def _outputs(net, fill):
    import torch
    return [torch.full((t.numel(),), fill, device="cuda") for t in (net.grid, net.weights, net.biases)]


@pytest.mark.parametrize("shape", ["cfg1", "cfg2"])
def test_static_backward_matches_oracle_twice(srn, shape):
    import torch
    S = srn
    if shape == "cfg1":
        p = H.cfg1_params(seed=50)
        n = 1 << 18  # the fit's batch of the plain workload fits the static array
    else:
        p = H.cfg2_params(seed=51, R=32)
        n = 100_003  # ragged against the 128-point blocks and the 2048-key sort blocks
    net = S.Network(p, max_fit_points=n)
    rng = np.random.default_rng(52)
    pts_np = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    pts_np[:3] = [[0, 0, 0], [1, 1, 1], [0.5, 1, 0]]
    dout_np = rng.normal(size=(n, net.out_dim)).astype(np.float32)
    pts = torch.tensor(pts_np, device="cuda")
    dout = torch.tensor(dout_np, device="cuda")
    rW, rb, rg = oracle.net_backward(oracle.OracleNet(p), pts_np, dout_np)
    ref = [rg, np.concatenate([w.ravel() for w in rW]), np.concatenate(rb)]
    ctx_out = _outputs(net, 0.0)
    S.srn_backward(net.ctx, pts, dout, *ctx_out)
    torch.cuda.synchronize()
    first = None
    for call in range(2):
        got = _outputs(net, float("nan"))
        S.srn_backward_static(net.cfg, net._params(), pts, dout, *got)
        torch.cuda.synchronize()
        for name, g, r, c in zip(("grid", "weights", "biases"), got, ref, ctx_out):
            g = g.cpu().numpy()
            err = _rel(g, r)
            print(f"{shape} call {call} d{name}: error vs FP64 {err:.2e} (relative to the block maximum)")
            assert err <= TOL_GRAD, (shape, call, name, err)
            assert _rel(g, c.cpu().numpy()) <= TOL_GRAD, (shape, call, name)
        if first is None:
            first = [g.clone() for g in got]
        else:  # deterministic: the second call repeats the first bit for bit
            assert all(torch.equal(a, b) for a, b in zip(first, got))
    net.close()


def test_static_backward_allocates_nothing(srn):
    """After the first call on the device (which looks up the array's
    address), a call leaves torch's allocator and the device's free memory
    untouched."""
    import torch
    S = srn
    p = H.cfg1_params(seed=54)
    n = 50_000
    net = S.Network(p)
    rng = np.random.default_rng(55)
    pts = torch.tensor(rng.uniform(0, 1, (n, 3)).astype(np.float32), device="cuda")
    dout = torch.tensor(rng.normal(size=(n, 1)).astype(np.float32), device="cuda")
    got = _outputs(net, 0.0)
    S.srn_backward_static(net.cfg, net._params(), pts, dout, *got)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        S.srn_backward_static(net.cfg, net._params(), pts, dout, *got)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0, (free0, free1)
    net.close()


def test_static_backward_empty_batch_zeroes_outputs(srn):
    """n = 0: no points, so every gradient is zero (outputs start as NaN)."""
    import torch
    S = srn
    p = H.cfg2_params(seed=56, R=16)
    net = S.Network(p)
    got = _outputs(net, float("nan"))
    S.srn_backward_static(net.cfg, net._params(), torch.zeros((0, 3), device="cuda"),
                          torch.zeros((0, 1), device="cuda"), *got)
    torch.cuda.synchronize()
    for g in got:
        assert bool(torch.all(g == 0)), "an output of the empty batch is not zero"
    net.close()


def test_static_backward_rejects_oversized_batches(srn):
    import torch
    S = srn
    p = H.cfg2_params(seed=53, R=32)
    net = S.Network(p)
    n = 1 << 20
    pts = torch.zeros((n, 3), device="cuda")
    dout = torch.zeros((n, 1), device="cuda")
    outs = _outputs(net, 0.0)
    with pytest.raises(S.SrnError) as e:
        S.srn_backward_static(net.cfg, net._params(), pts, dout, *outs)
    assert e.value.status == S.SRN_ERR_INVALID_ARG
    assert "static area" in str(e.value) and "at most n" in str(e.value)
    net.close()
