"""GPU parity of the wider networks of the width / layer sweep (Section 4.1
performance figure; Section 6.1 grid ablation): hidden width 48 and 64 with
2 to 6 layers, on the FP32 CUDA-core path and the FP16 tensor-core path.

The input vector is widened with the hidden width as in the 32-channel
network (3 + 2m + F + 1 padding = c + 16 with F = 16): m = 22 Fourier rows
for c = 48, m = 30 for c = 64."""
import numpy as np
import pytest

import oracle
from paper_2112_01579_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

M_FOR = {c: synth.fourier_rows_for_width(c) for c in (32, 48, 64)}


@pytest.fixture(scope="module")
def srn():
    import torch
    from paper_2112_01579_gb300 import build
    build.build()
    from paper_2112_01579_gb300 import srn as S
    assert torch.cuda.is_available()
    return S


def _params(width, layers, seed, R=16):
    return synth.random_params(R=R, F=16, m=M_FOR[width], layers=layers, width=width, act=synth.ACT_SNAKEALT,
                               seed=seed, grid_std=0.5, bias_std=0.2)


def _render(S, net, cams, tf, W, Hh, step, et):
    import torch
    out = torch.full((1, len(cams), Hh, W, 4), -1.0, device="cuda")
    S.srn_render(net.ctx, cams, tf, S.render_desc(W, Hh, step, et), out)
    torch.cuda.synchronize()
    st, msg = S.srn_sync_status(net.ctx)
    assert st == 0, msg
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("width,layers", [(48, 2), (48, 4), (48, 6), (64, 2), (64, 4), (64, 6)])
def test_wide_render_parity(srn, width, layers, precision):
    """Two views of 40 x 36 pixels (a ragged 8 x 4 pixel-tile edge; several
    128-ray tiles) at step 1/128 with early termination."""
    S = srn
    p = _params(width, layers, 300 + 10 * width + layers)
    q = synth.to_half_exact(p) if precision else p
    net = S.Network(q, precision=precision)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    got = _render(S, net, cams, tf, 40, 36, 1 / 128, 0.99)
    on = oracle.OracleNet(q)
    ref, mg, _ = oracle.render(on, cams, H.oracle_tf(tf), 40, 36, 1 / 128, 0.99, want_margin=True)
    tol = H.TOL_FP16_IMG if precision else H.TOL_FP32_IMG
    r = H.compare_images(got, ref, mg, tol, 0.99)
    print(f"width {width} x {layers} precision {precision}: max error {r['max_strict']:.2e}, "
          f"worst error / bound {r['worst_ratio']:.2f}")
    assert r["ok"], r


@pytest.mark.parametrize("width,layers", [(48, 3), (64, 5)])
def test_wide_eval_parity(srn, width, layers):
    """Density at 50,000 random points: FP16 tensor-core layers against the
    oracle on the FP16-rounded parameters, and the FP32 path's density and
    adjoint input gradient against the oracle."""
    import torch
    S = srn
    p = _params(width, layers, 400 + width + layers)
    pts = np.random.default_rng(401).uniform(0, 1, (50000, 3)).astype(np.float32)
    q = synth.to_half_exact(p)
    n16 = S.Network(q, precision=S.SRN_PREC_FP16)
    o = torch.zeros((len(pts), 1), device="cuda")
    S.srn_eval(n16.ctx, torch.tensor(pts, device="cuda"), o)
    torch.cuda.synchronize()
    err = H.rel_density_err(o.cpu().numpy(), oracle.net_forward(oracle.OracleNet(q), pts))
    assert err.max() <= H.TOL_FP16_RHO, err.max()

    n32 = S.Network(p)
    on = oracle.OracleNet(p)
    rho = torch.zeros(len(pts), device="cuda")
    grad = torch.zeros((len(pts), 3), device="cuda")
    S.srn_density_grad(n32.ctx, torch.tensor(pts, device="cuda"), rho, grad)
    torch.cuda.synchronize()
    ref_rho, ref_g = oracle.net_input_grad(on, pts)
    assert H.rel_density_err(rho.cpu().numpy(), ref_rho.reshape(-1)).max() <= H.TOL_FP32_RHO
    g = grad.cpu().numpy()
    B = oracle.error_bounds(on, pts, oracle.PREC_FP32)[1]  # first-order bound of the FP32 gradient error
    assert np.all(np.abs(g - ref_g) <= B), (np.abs(g - ref_g) / B).max()


@pytest.mark.parametrize("width", [48, 64])
@pytest.mark.parametrize("shading", [1, 2, 3])
def test_wide_shading_parity(srn, width, shading):
    """Section 5 shading on the wider networks, tensor-core path: adjoint
    (backward MMAs with the wider accumulator and derivative stash), central
    differences and the 4-output head, against the oracle within the FP16
    image bound plus the derived shading allowance."""
    S = srn
    p = synth.random_params(R=12, F=16, m=M_FOR[width], layers=4 if shading == 1 else 3, width=width,
                            out_dim=4 if shading == 3 else 1, act=synth.ACT_SNAKEALT, seed=410 + width + shading,
                            grid_std=0.5, bias_std=0.2)
    q = synth.to_half_exact(p)
    net = S.Network(q, precision=S.SRN_PREC_FP16)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(1)
    import torch
    out = torch.full((1, 1, 16, 24, 4), -1.0, device="cuda")  # small: the adjoint bound costs ~400 passes a sample
    S.srn_render(net.ctx, cams, tf, S.render_desc(24, 16, 1 / 48, 2.0, shading, 1 / 64), out)
    torch.cuda.synchronize()
    assert S.srn_sync_status(net.ctx)[0] == 0
    ref, bound = oracle.render_shade_bound(oracle.OracleNet(q), cams, H.oracle_tf(tf), 24, 16, 1 / 48, 2.0, shading,
                                           oracle.PREC_FP16, fd_h=1 / 64)
    r = H.compare_images(out.cpu().numpy()[0], ref[0], None, H.shaded_tol(H.TOL_FP16_IMG, bound[0]), 2.0)
    print(f"width {width} shading {shading}: max error {r['max_strict']:.2e}, worst error / bound "
          f"{r['worst_ratio']:.2f}")
    assert r["ok"], r


def test_wide_unsupported_shapes_fail_loudly(srn):
    """The tensor-core variants of width 48 / 64 cover SnakeAlt, 16 latent
    channels and the widened Fourier count, every shading mode; other shapes
    and the fused fit (width 32 only) return SRN_ERR_UNSUPPORTED."""
    import torch
    S = srn
    p = synth.to_half_exact(synth.random_params(R=8, F=16, m=22, layers=3, width=48, act=synth.ACT_SINE, seed=402))
    net = S.Network(p, precision=S.SRN_PREC_FP16)
    out = torch.zeros((1, 1, 8, 8, 4), device="cuda")
    with pytest.raises(S.SrnError) as e:
        S.srn_render(net.ctx, synth.orbit_cameras(1), synth.tf_preset(4), S.render_desc(8, 8, 0.01), out)
    assert e.value.status == S.SRN_ERR_UNSUPPORTED
    p = _params(64, 5, 403, R=8)  # five layers: beyond the adjoint's TMEM layout
    net = S.Network(synth.to_half_exact(p), precision=S.SRN_PREC_FP16)
    with pytest.raises(S.SrnError) as e:
        S.srn_render(net.ctx, synth.orbit_cameras(1), synth.tf_preset(4), S.render_desc(8, 8, 0.01, 0.99, 1), out)
    assert e.value.status == S.SRN_ERR_UNSUPPORTED
    fit = S.Network(p, max_fit_points=1024, adam=True)
    vol = torch.zeros((16, 16, 16), device="cuda")
    with pytest.raises(S.SrnError) as e:
        S.srn_fit_step(fit.ctx, vol, 1024, 1, 0, torch.zeros(1, device="cuda"))
    assert e.value.status == S.SRN_ERR_UNSUPPORTED
