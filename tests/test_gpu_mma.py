"""GPU parity of the FP16 tensor-core render (tcgen05 / TMEM) against the FP64
oracle evaluated with the same FP16 parameter values, through the C ABI."""
import math

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


def _net16(S, p):
    q = synth.to_half_exact(p)
    net = S.Network(q, precision=S.SRN_PREC_FP16)
    return net, q


def _render(S, net, cams, tf, W, Hh, step, et, shading=0, fd_h=0.0, times=None):
    import torch
    T = 1 if times is None else len(times)
    out = torch.full((T, len(cams), Hh, W, 4), -1.0, device="cuda")
    ns = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.srn_render(net.ctx, cams, tf, S.render_desc(W, Hh, step, et, shading, fd_h), out, times=times, samples=ns)
    torch.cuda.synchronize()
    st, msg = S.srn_sync_status(net.ctx)
    assert st == 0, msg
    return out.cpu().numpy(), int(ns.item())


@pytest.mark.parametrize("et", [2.0, 0.99])
def test_mma_cfg2_network_small_frames(srn, et):
    S = srn
    net, q = _net16(S, H.cfg2_params(seed=20))
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    got, ns = _render(S, net, cams, tf, 64, 48, 1 / 128, et)
    ref, mg, ns_ref = oracle.render(oracle.OracleNet(q), cams, H.oracle_tf(tf), 64, 48, 1 / 128, et,
                                    want_margin=True)
    assert np.all(got >= 0)  # every pixel written
    r = H.compare_images(got[0], ref[0], mg[0], H.TOL_FP16_IMG, et)
    assert r["ok"], r
    assert abs(ns - ns_ref) <= 0.002 * ns_ref + 2
    assert ref[0, ..., 3].max() > 0.2


def test_mma_cfg1_shape_sine(srn):
    S = srn
    net, q = _net16(S, H.cfg1_params(seed=21))
    tf = synth.tf_preset(4)
    cams = synth.orbit_cameras(3)
    got, _ = _render(S, net, cams, tf, 40, 40, 1 / 128, 2.0)
    ref, _, _ = oracle.render(oracle.OracleNet(q), cams, H.oracle_tf(tf), 40, 40, 1 / 128, 2.0)
    assert np.abs(got[0] - ref[0]).max() <= H.TOL_FP16_IMG


def test_mma_ragged_and_degenerate_images(srn):
    S = srn
    net, q = _net16(S, H.cfg2_params(seed=22))
    tf = synth.tf_preset(8)
    cams = [dict(eye=[0.9, 0.3, 0.9], target=[0.5, 0.6, 0.0], up=[0, 1, 0], fovy=math.radians(70))]
    for W, Hh in [(37, 23), (1, 1), (9, 5), (130, 3)]:
        got, _ = _render(S, net, cams, tf, W, Hh, 1 / 100, 2.0)
        ref, _, _ = oracle.render(oracle.OracleNet(q), cams, H.oracle_tf(tf), W, Hh, 1 / 100, 2.0)
        assert np.all(got >= 0)
        assert np.abs(got - ref).max() <= H.TOL_FP16_IMG, (W, Hh)
    miss = [dict(eye=[0, 0, 3], target=[0, 0, 6], up=[0, 1, 0], fovy=0.5)]
    got, ns = _render(S, net, miss, tf, 16, 16, 1 / 100, 0.99)
    assert ns == 0 and np.all(got == 0)


def test_mma_full_size_sampled_pixels(srn):
    """Config 2 launch configuration: 1024 x 1024, step 1/512, ET 0.99."""
    S = srn
    net, q = _net16(S, H.cfg2_params(seed=23))
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(1)
    got, ns = _render(S, net, cams, tf, 1024, 1024, 1 / 512, 0.99)
    assert np.all(got >= 0)
    pix = synth.sample_pixels(1, 1, 1024, 1024, 300, seed=24)
    ref, mg, _ = oracle.render(oracle.OracleNet(q), cams, H.oracle_tf(tf), 1024, 1024, 1 / 512, 0.99, pixels=pix,
                               want_margin=True)
    r = H.compare_images(got.reshape(-1, 4)[pix], ref, mg, H.TOL_FP16_IMG, 0.99)
    assert r["ok"], r


def test_mma_matches_fp32_path_sample_count(srn):
    """Same network (FP16-exact values) in both precisions: the number of
    network samples of a frame without early termination agrees to the
    handful of rays whose last segment rounds differently."""
    import torch
    S = srn
    q = synth.to_half_exact(H.cfg2_params(seed=25))
    n16 = S.Network(q, precision=S.SRN_PREC_FP16)
    n32 = S.Network(q, precision=S.SRN_PREC_FP32)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(1)
    a, na = _render(S, n16, cams, tf, 256, 256, 1 / 256, 2.0)
    b, nb = _render(S, n32, cams, tf, 256, 256, 1 / 256, 2.0)
    assert abs(na - nb) <= 0.001 * nb
    assert np.abs(a - b).max() <= H.TOL_FP16_IMG


@pytest.mark.parametrize("shading", [1, 2, 3])
def test_mma_shading(srn, shading):
    S = srn
    net, q = _net16(S, H.cfg2_params(seed=26, R=16, out_dim=4 if shading == 3 else 1))
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    got, _ = _render(S, net, cams, tf, 32, 24, 1 / 64, 2.0, shading=shading, fd_h=1 / 64)
    ref, bound = oracle.render_shade_bound(oracle.OracleNet(q), cams, H.oracle_tf(tf), 32, 24, 1 / 64, 2.0, shading,
                                           oracle.PREC_FP16, fd_h=1 / 64)
    # per pixel: the FP16 image bound plus what the FP16 path's gradient error
    # bound (central differences: density bounds over 2h; head: output
    # bounds; adjoint: its gradient bound) moves through the shading formula
    r = H.compare_images(got[0], ref[0], None, H.shaded_tol(H.TOL_FP16_IMG, bound[0]), 2.0)
    print(f"fp16 shading {shading}: max error {r['max_strict']:.2e}, worst error / bound {r['worst_ratio']:.2f}")
    assert r["ok"], r


@pytest.mark.parametrize("shape", ["cfg1_sine_l2", "snake_l3"])
def test_mma_adjoint_shapes(srn, shape):
    """The tensor-core adjoint (backward MMAs through W_h^T and W_0^T) on the
    other instantiated shapes: 12 Fourier rows / 8 channels with sine and two
    layers (no hidden backward), and three SnakeAlt layers (one)."""
    S = srn
    if shape == "cfg1_sine_l2":
        p = H.cfg1_params(seed=27)
    else:
        p = synth.random_params(R=12, F=16, m=14, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=28,
                                grid_std=0.5, bias_std=0.2)
    net, q = _net16(S, p)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    got, _ = _render(S, net, cams, tf, 40, 28, 1 / 64, 2.0, shading=1)
    ref, bound = oracle.render_shade_bound(oracle.OracleNet(q), cams, H.oracle_tf(tf), 40, 28, 1 / 64, 2.0, 1,
                                           oracle.PREC_FP16)
    r = H.compare_images(got[0], ref[0], None, H.shaded_tol(H.TOL_FP16_IMG, bound[0]), 2.0)
    assert r["ok"], r


@pytest.mark.parametrize("shape", ["cfg1", "cfg2", "snake_l3", "init_cfg2", "keyframes", "head", "w48", "w64"])
def test_mma_adjoint_gradient_matches_oracle(srn, shape):
    """srn_density_grad on an FP16 context runs the tensor-core adjoint (the
    render's backward MMAs, Section 5 "adjoint") at given points: the density
    within the FP16 bound and every gradient component within its
    first-order error bound for the FP16 path (oracle.fp16_grad_bound: the
    layer-0 inputs rounded to FP16, MUFU activations and derivatives, hi + lo
    hidden and adjoint rows, FP32 accumulation and Jacobians), element by
    element, 20,000 points including faces and corners."""
    import torch
    S = srn
    t = 0.0
    if shape == "cfg1":
        p = H.cfg1_params(seed=90)
    elif shape == "cfg2":
        p = H.cfg2_params(seed=91)
    elif shape == "snake_l3":
        p = synth.random_params(R=12, F=16, m=14, layers=3, width=32, act=synth.ACT_SNAKEALT, seed=92,
                                grid_std=0.5, bias_std=0.2)
    elif shape == "init_cfg2":
        p = synth.init_params(R=32, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=0)
    elif shape == "keyframes":
        p = H.cfg2_params(seed=93, R=12, nkey=3, key_times=[0.0, 1.0, 3.0])
        t = 1.6
    elif shape == "head":  # the gradient of output 0 of a 4-output network
        p = H.cfg2_params(seed=95, R=12, out_dim=4)
    else:  # the sweep's wider networks: widths 48 / 64, 22 / 30 Fourier rows
        c = 48 if shape == "w48" else 64
        p = synth.random_params(R=12, F=16, m=synth.fourier_rows_for_width(c), layers=4, width=c,
                                act=synth.ACT_SNAKEALT, seed=96 + c, grid_std=0.5, bias_std=0.2)
    net, q = _net16(S, p)
    on = oracle.OracleNet(q)
    n = 20000
    pts = np.random.default_rng(94).uniform(0, 1, (n, 3)).astype(np.float32)
    pts[:4] = [[0, 0, 0], [1, 1, 1], [0.5, 1.0, 0.0], [1e-7, 0.999999, 0.5]]
    rho = torch.zeros(n, device="cuda")
    g = torch.zeros((n, 3), device="cuda")
    S.srn_density_grad(net.ctx, torch.tensor(pts, device="cuda"), rho, g, time=t)
    torch.cuda.synchronize()
    assert S.srn_sync_status(net.ctx)[0] == S.SRN_OK
    r2, g2 = oracle.net_input_grad(on, pts, t)
    err_rho = H.rel_density_err(rho.cpu().numpy(), r2).max()
    print(f"fp16 adjoint {shape}: max rel density error {err_rho:.2e}")
    assert err_rho <= H.TOL_FP16_RHO, err_rho
    B = oracle.error_bounds(on, pts, oracle.PREC_FP16, t)[1]
    diff = np.abs(g.cpu().numpy().astype(np.float64) - g2)
    gs = np.maximum(np.abs(g2).max(axis=1), 1.0)
    print(f"fp16 adjoint {shape}: worst error / bound {(diff / B).max():.2f}, max error / max(|g|, 1) "
          f"{(diff.max(axis=1) / gs).max():.2e}")
    assert np.all(diff <= B), (diff / B).max()


def test_mma_adjoint_limits(srn):
    """Five layers (three stashed derivative blocks, beyond the TMEM layout)
    or a direct time input: the tensor-core adjoint refuses with
    SRN_ERR_UNSUPPORTED, for shading and for srn_density_grad."""
    import torch
    S = srn
    out = torch.zeros((1, 1, 8, 8, 4), device="cuda")
    for p in (synth.random_params(R=8, F=16, m=14, layers=5, width=32, act=synth.ACT_SNAKEALT, seed=29),
              synth.random_params(R=8, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=31,
                                  n_keyframes=2, key_times=[0.0, 1.0], time_input=1)):
        net, _ = _net16(S, p)
        with pytest.raises(S.SrnError) as e:
            S.srn_render(net.ctx, synth.orbit_cameras(1), synth.tf_preset(4), S.render_desc(8, 8, 0.01, 2.0, 1), out)
        assert e.value.status == S.SRN_ERR_UNSUPPORTED
        with pytest.raises(S.SrnError) as e:
            S.srn_density_grad(net.ctx, torch.zeros((4, 3), device="cuda"), torch.zeros(4, device="cuda"),
                               torch.zeros((4, 3), device="cuda"))
        assert e.value.status == S.SRN_ERR_UNSUPPORTED


def test_mma_time_batch(srn):
    """Config 5 layout at small size: 5 keyframes (0, 4, 8, 12, 15), 16 times x
    4 views in one launch."""
    S = srn
    p = H.cfg2_params(seed=27, R=16, nkey=5, key_times=[0, 4, 8, 12, 15])
    net, q = _net16(S, p)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(4)
    times = list(range(16))
    got, _ = _render(S, net, cams, tf, 20, 12, 1 / 64, 0.99, times=times)
    ref, mg, _ = oracle.render(oracle.OracleNet(q), cams, H.oracle_tf(tf), 20, 12, 1 / 64, 0.99, times=times,
                               want_margin=True)
    r = H.compare_images(got, ref, mg, H.TOL_FP16_IMG, 0.99)
    assert r["ok"], r


@pytest.mark.parametrize("grid_u8", [False, True])
def test_mma_fp16_latent_grid_scaling(srn, grid_u8):
    """A latent grid beyond the FP16 range (values to ~3e5, FP16 stops at
    65504) whose layer-0 weights are correspondingly small, so the network
    itself is well conditioned: the FP16 copy holds G 2^-k (k chosen from
    max |G| by srn_sync_half) and the latent columns' weights are staged
    times 2^k, exactly.  Render, point evaluation and the tensor-core
    adjoint match the oracle within the FP16 bounds; the 8-bit grid applies
    the same scale to its per-channel lo / step."""
    import torch
    S = srn
    p = synth.to_half_exact(H.cfg2_params(seed=29, R=8))
    p["grid"] = (p["grid"] * 2.0 ** 17).astype(np.float32)  # FP16 values times 2^17: G 2^-k stays FP16-exact
    W0 = p["weights"][0].copy()
    lat = slice(3 + 28, 3 + 28 + 16)
    # the latent columns times 2^-17, rounded to FP16 (subnormals): the values the FP16 copy holds
    W0[:, lat] = (W0[:, lat] * 2.0 ** -17).astype(np.float16).astype(np.float32)
    p["weights"] = [W0] + p["weights"][1:]
    assert np.abs(p["grid"]).max() > 65504
    on = oracle.OracleNet(p)
    net = S.Network(p, precision=S.SRN_PREC_FP16, grid_u8=grid_u8)
    tf, cams = synth.tf_preset(8), synth.orbit_cameras(2)
    got, _ = _render(S, net, cams, tf, 40, 28, 1 / 64, 0.99)
    assert S.srn_sync_status(net.ctx)[0] == S.SRN_OK
    oq = oracle.OracleNet(H.u8_params(p)) if grid_u8 else on
    ref, mg, _ = oracle.render(oq, cams, H.oracle_tf(tf), 40, 28, 1 / 64, 0.99, want_margin=True)
    r = H.compare_images(got[0], ref[0], mg[0], H.TOL_FP16_IMG, 0.99)
    assert r["ok"], r
    pts = np.random.default_rng(31).uniform(0, 1, (20000, 3)).astype(np.float32)
    err = H.rel_density_err(_eval16(S, net, pts), oracle.net_forward(oq, pts))
    assert err.max() <= H.TOL_FP16_RHO, err.max()
    if not grid_u8:
        rho = torch.zeros(len(pts), device="cuda")
        g = torch.zeros((len(pts), 3), device="cuda")
        S.srn_density_grad(net.ctx, torch.tensor(pts, device="cuda"), rho, g)
        torch.cuda.synchronize()
        r2, g2 = oracle.net_input_grad(on, pts)
        assert H.rel_density_err(rho.cpu().numpy(), r2).max() <= H.TOL_FP16_RHO
        B = oracle.fp16_grad_bound(on, pts)
        assert np.all(np.abs(g.cpu().numpy() - g2) <= B), np.max(np.abs(g.cpu().numpy() - g2) / B)


def test_mma_fp16_overflow_is_reported(srn):
    """Activations beyond the FP16 range are reported, not scaled: a hidden
    activation above 65504 needs a pre-activation |x| > 1.3e5, whose FP32
    rounding alone (|x| 2^-24 > 0.007) moves sin x by more than the image
    bound, so no FP32-accumulating kernel evaluates such a network within
    tolerance.  Here the latent grid (values to 4e7) is scaled into FP16 but
    the hidden activations overflow: the tensor-core render reports
    SRN_ERR_NONFINITE; the FP32 path renders the same network with finite
    values; a normal network leaves the status at SRN_OK."""
    import torch
    S = srn
    p = H.cfg2_params(seed=29, R=8)
    p["grid"] = (p["grid"] * 2e7).astype(np.float32)
    tf, cams = synth.tf_preset(8), synth.orbit_cameras(1)
    out = torch.zeros((1, 1, 16, 16, 4), device="cuda")
    n16 = S.Network(p, precision=S.SRN_PREC_FP16)
    S.srn_render(n16.ctx, cams, tf, S.render_desc(16, 16, 1 / 64, 2.0), out)
    st, _ = S.srn_sync_status(n16.ctx)
    assert st == S.SRN_ERR_NONFINITE
    assert S.srn_sync_status(n16.ctx)[0] == S.SRN_OK  # reading clears it
    n32 = S.Network(p, precision=S.SRN_PREC_FP32)
    S.srn_render(n32.ctx, cams, tf, S.render_desc(16, 16, 1 / 64, 2.0), out)
    assert S.srn_sync_status(n32.ctx)[0] == S.SRN_OK
    assert torch.isfinite(out).all()
    ok = S.Network(synth.to_half_exact(H.cfg2_params(seed=30, R=8)), precision=S.SRN_PREC_FP16)
    S.srn_render(ok.ctx, cams, tf, S.render_desc(16, 16, 1 / 64, 2.0), out)
    assert S.srn_sync_status(ok.ctx)[0] == S.SRN_OK


def test_mma_rejects_unsupported(srn):
    S = srn
    p = synth.random_params(R=8, F=12, m=10, layers=3, width=32, seed=28)
    q = synth.to_half_exact(p)
    with pytest.raises(S.SrnError) as e:
        net = S.Network(q, precision=S.SRN_PREC_FP16)
        import torch
        out = torch.zeros((1, 1, 8, 8, 4), device="cuda")
        S.srn_render(net.ctx, synth.orbit_cameras(1), synth.tf_preset(4), S.render_desc(8, 8, 0.01), out)
    assert e.value.status == S.SRN_ERR_UNSUPPORTED


def _eval16(S, net, pts, t=0.0):
    import torch
    out = torch.zeros((len(pts), net.out_dim), device="cuda")
    S.srn_eval(net.ctx, torch.tensor(pts, device="cuda"), out, time=t)
    torch.cuda.synchronize()
    st, msg = S.srn_sync_status(net.ctx)
    assert st == 0, msg
    return out.cpu().numpy()


@pytest.mark.parametrize("shape", ["cfg2", "cfg1", "head", "time"])
def test_mma_eval_density_parity(srn, shape):
    """FP16 tensor-core network at points vs the FP64 oracle on the same FP16
    parameters: relative density error <= 1e-3."""
    S = srn
    t = 0.0
    if shape == "cfg2":
        p = H.cfg2_params(seed=60)
    elif shape == "cfg1":
        p = H.cfg1_params(seed=61)
    elif shape == "head":
        p = H.cfg2_params(seed=62, R=16, out_dim=4)
    else:
        p = H.cfg2_params(seed=63, R=16, nkey=5, key_times=[0, 4, 8, 12, 15])
        t = 9.5
    net, q = _net16(S, p)
    rng = np.random.default_rng(64)
    n = 100_003  # ragged against the 128-row tiles
    pts = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    pts[:4] = [[0, 0, 0], [1, 1, 1], [0.5, 1, 0], [1e-7, 0.999999, 0.5]]
    got = _eval16(S, net, pts, t)
    ref = oracle.net_forward(oracle.OracleNet(q), pts, t)
    err = H.rel_density_err(got, ref)
    print(f"fp16 eval {shape}: max rel density error {err.max():.2e}, mean {err.mean():.2e}")
    assert err.max() <= H.TOL_FP16_RHO


def test_mma_eval_trained_network(srn):
    """The same check on a trained network (weights and grid move away from
    their initial ranges during training): trained by the oracle's FP64 fit,
    rounded to FP16."""
    S = srn
    vol = synth.noise_volume(48, seed=65).numpy()
    p = synth.init_params(R=16, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=66)
    q = H.oracle_trained_params(vol, p)
    net = S.Network(q, precision=S.SRN_PREC_FP16)
    pts = np.random.default_rng(67).uniform(0, 1, (20000, 3)).astype(np.float32)
    got = _eval16(S, net, pts)
    ref = oracle.net_forward(oracle.OracleNet(q), pts)
    err = H.rel_density_err(got, ref)
    print(f"fp16 eval trained: max rel density error {err.max():.2e}, mean {err.mean():.2e}")
    assert err.max() <= H.TOL_FP16_RHO


@pytest.mark.parametrize("which", ["cfg1", "cfg2"])
def test_mma_bounded_wait_reports_timeout(srn, monkeypatch, which):
    """The timeout path without a fault: with SRN_TEST_STALL=1 the render
    issues no MMA (nothing in flight), every warpgroup's bounded mbarrier
    wait runs out after about a second, the kernel frees its TMEM and returns,
    and the status reads SRN_ERR_TIMEOUT; the context then renders normally."""
    import time
    import torch
    S = srn
    net, q = _net16(S, H.cfg1_params(seed=23) if which == "cfg1" else H.cfg2_params(seed=24, R=16))
    tf = synth.tf_preset(4)
    cams = synth.orbit_cameras(1)
    out = torch.full((1, 1, 16, 16, 4), -1.0, device="cuda")
    torch.cuda.synchronize()
    monkeypatch.setenv("SRN_TEST_STALL", "1")
    t0 = time.time()
    S.srn_render(net.ctx, cams, tf, S.render_desc(16, 16, 1 / 64, 0.99), out)
    torch.cuda.synchronize()
    dt = time.time() - t0
    monkeypatch.delenv("SRN_TEST_STALL")
    st, msg = S.srn_sync_status(net.ctx)
    assert st == S.SRN_ERR_TIMEOUT, (st, msg)
    assert 0.2 < dt < 60, dt
    got, _ = _render(S, net, cams, tf, 16, 16, 1 / 64, 2.0)
    ref, _, _ = oracle.render(oracle.OracleNet(q), cams, H.oracle_tf(tf), 16, 16, 1 / 64, 2.0)
    assert np.abs(got - ref).max() <= H.TOL_FP16_IMG
    net.close()


def test_mma_single_grid_kernel_equals_keyframe_kernel(srn):
    """The render instantiation for one latent grid (no time blend) against
    the keyframe instantiation on the same grid stored as two identical
    keyframes, rendered at the first keyframe time: the blend weights are
    exactly 1 and 0, so the two images agree bit for bit; both against the
    oracle at the FP16 bound."""
    import torch
    S = srn
    p1 = H.cfg2_params(seed=97, R=16)
    p2 = dict(p1)
    p2["grid"] = np.concatenate([p1["grid"], p1["grid"]], axis=0)  # [keyframe][z][y][x][F]
    p2["key_times"] = np.asarray([0.0, 1.0], np.float32)
    n1, q1 = _net16(S, p1)
    n2, _ = _net16(S, p2)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    a, _ = _render(S, n1, cams, tf, 48, 40, 1 / 128, 0.99)
    b, _ = _render(S, n2, cams, tf, 48, 40, 1 / 128, 0.99, times=[0.0])
    assert np.array_equal(a, b)
    ref, mg, _ = oracle.render(oracle.OracleNet(q1), cams, H.oracle_tf(tf), 48, 40, 1 / 128, 0.99, want_margin=True)
    r = H.compare_images(a[0], ref[0], mg[0], H.TOL_FP16_IMG, 0.99)
    assert r["ok"], r
    n1.close()
    n2.close()
