"""srn_backward_static: the parameter backward for callers that cannot
allocate device memory.

Some integrations may not call cudaMalloc at all: code running while a
stream is captured into a CUDA graph, hosts whose device memory belongs to
another allocator, or frame loops that must not take the device
synchronization an allocation can cause.  srn_backward needs a context
(srn_create allocates its scratch); srn_backward_static takes the network
description directly and works in a fixed device area inside the library.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes alone in a fresh
process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2112_01579_gb300 import synth
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
    a, b = a.double().cpu().numpy().ravel(), b.double().cpu().numpy().ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("shape", ["cfg1", "cfg2"])
def test_static_backward_matches_context_backward_twice(srn, shape):
    import torch
    S = srn
    if shape == "cfg1":
        p = H.cfg1_params(seed=50)
        n = 1 << 18  # the fit's batch of the plain workload fits the static area
    else:
        p = H.cfg2_params(seed=51, R=32)
        n = 100_000
    net = S.Network(p, max_fit_points=n)
    rng = np.random.default_rng(52)
    pts = torch.tensor(rng.uniform(0, 1, (n, 3)).astype(np.float32), device="cuda")
    dout = torch.tensor(rng.normal(size=(n, net.out_dim)).astype(np.float32), device="cuda")
    ref = [torch.empty(net.grid.numel(), device="cuda"), torch.empty(net.weights.numel(), device="cuda"),
           torch.empty(net.biases.numel(), device="cuda")]
    S.srn_backward(net.ctx, pts, dout, *ref)
    for call in range(2):  # the second call reuses the area the first one left behind
        got = [torch.full_like(r, float("nan")) for r in ref]
        S.srn_backward_static(net.cfg, net._params(), pts, dout, *got)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert _rel(g, r) <= TOL_GRAD, (shape, call)


def test_static_backward_rejects_oversized_batches(srn):
    import torch
    S = srn
    p = H.cfg2_params(seed=53, R=32)
    net = S.Network(p)
    n = 1 << 20
    pts = torch.zeros((n, 3), device="cuda")
    dout = torch.zeros((n, 1), device="cuda")
    outs = [torch.empty(net.grid.numel(), device="cuda"), torch.empty(net.weights.numel(), device="cuda"),
            torch.empty(net.biases.numel(), device="cuda")]
    with pytest.raises(S.SrnError) as e:
        S.srn_backward_static(net.cfg, net._params(), pts, dout, *outs)
    assert e.value.status == S.SRN_ERR_INVALID_ARG
    assert "static area" in str(e.value) and "at most n" in str(e.value)
