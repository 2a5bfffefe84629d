"""torch.autograd binding of the fV-SRN network.

``SRNFunction`` runs the forward pass with ``srn_eval`` and the backward pass
with the library's hand-written kernels: ``srn_backward`` for the latent grid
(atomic-free gather over points sorted by cell), weights and biases, and
``srn_input_backward`` (the adjoint seeded with the incoming gradient) for the
input positions.  ``SRNModule`` owns the
parameters as ``nn.Parameter`` tensors so any torch optimizer can train the
network (``srn_fit_step`` is the fused alternative).  Marshalling only: no
computation happens in Python.
"""
from __future__ import annotations

import torch

from . import srn as S


class SRNFunction(torch.autograd.Function):
    """out[n, D] = network(pts[n, 3]) at time t.

    grid / weights / biases must be the tensors the context was created
    with (the kernels read them through the context); they are inputs here
    only so autograd routes their gradients."""

    @staticmethod
    def forward(ctx, pts, grid, weights, biases, net, time):
        pts = pts.contiguous()
        if net.cfg.precision == S.SRN_PREC_FP16:
            S.srn_sync_half(net.ctx)  # the FP16 copies follow the masters after each update
        out = torch.empty((pts.shape[0], net.out_dim), device=pts.device, dtype=torch.float32)
        S.srn_eval(net.ctx, pts, out, time=time)
        ctx.save_for_backward(pts)
        ctx.net, ctx.time = net, time
        return out

    @staticmethod
    def backward(ctx, dout):
        (pts,) = ctx.saved_tensors
        net = ctx.net
        dout = dout.contiguous().float()
        dgrid = dW = db = dpts = None
        if any(ctx.needs_input_grad[1:4]):
            dgrid = torch.empty_like(net.grid)
            dW = torch.empty_like(net.weights)
            db = torch.empty_like(net.biases)
            S.srn_backward(net.ctx, pts, dout, dgrid, dW, db, time=ctx.time)
        if ctx.needs_input_grad[0]:
            dpts = torch.empty((pts.shape[0], 3), device=pts.device)
            S.srn_input_backward(net.ctx, pts, dout, dpts, time=ctx.time)
        return dpts, dgrid, dW, db, None, None


class SRNModule(torch.nn.Module):
    """An fV-SRN whose parameters are torch Parameters on the GPU."""

    def __init__(self, params: dict, precision=S.SRN_PREC_FP32, max_batch=1 << 18):
        super().__init__()
        self.net = S.Network(params, precision=precision, max_fit_points=max_batch)
        self.grid = torch.nn.Parameter(self.net.grid, requires_grad=True)
        self.weights = torch.nn.Parameter(self.net.weights, requires_grad=True)
        self.biases = torch.nn.Parameter(self.net.biases, requires_grad=True)

    def forward(self, pts, time=0.0):
        return SRNFunction.apply(pts, self.grid, self.weights, self.biases, self.net, float(time))
