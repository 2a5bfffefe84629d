"""GPU parity of the FP32 CUDA-core path (render, dense DVR, eval, adjoint
gradient) against the FP64 oracle, through the C ABI."""
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


def _render_gpu(S, net, cams, tf, W, H_, step, et, shading=0, fd_h=0.0, times=None):
    import torch
    T = 1 if times is None else len(times)
    out = torch.zeros((T, len(cams), H_, W, 4), device="cuda")
    ns = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.srn_render(net.ctx, cams, tf, S.render_desc(W, H_, step, et, shading, fd_h), out, times=times, samples=ns)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(ns.item())


@pytest.mark.parametrize("et", [2.0, 0.99])
def test_render_fp32_cfg1_full_frame(srn, et):
    """Config 1 at its full size: 128 x 128, step 1/128, 4-point TF, two views."""
    S = srn
    p = H.cfg1_params(seed=0)
    net = S.Network(p)
    tf = synth.tf_preset(4)
    cams = synth.orbit_cameras(2)
    got, ns = _render_gpu(S, net, cams, tf, 128, 128, 1 / 128, et)
    ref, mg, ns_ref = oracle.render(oracle.OracleNet(p), cams, H.oracle_tf(tf), 128, 128, 1 / 128, et,
                                    want_margin=True)
    r = H.compare_images(got[0], ref[0], mg[0], H.TOL_FP32_IMG, et)
    assert r["ok"], r
    assert np.abs(ns - ns_ref) <= 0.001 * ns_ref
    assert ref[0, ..., 3].max() > 0.3  # the frame is not empty


def test_render_fp32_ragged_sizes_and_misses(srn):
    """Image sizes that do not fill the 8 x 4 warp tiles, a camera whose
    view misses the box partly, and a 1 x 1 image."""
    S = srn
    p = H.cfg1_params(seed=1)
    net = S.Network(p)
    tf = synth.tf_preset(4)
    cams = [dict(eye=[0.9, 0.3, 0.9], target=[0.5, 0.6, 0.0], up=[0, 1, 0], fovy=math.radians(70))]
    for W, Hh in [(37, 23), (1, 1), (9, 5)]:
        got, _ = _render_gpu(S, net, cams, tf, W, Hh, 1 / 100, 2.0)
        ref, _, _ = oracle.render(oracle.OracleNet(p), cams, H.oracle_tf(tf), W, Hh, 1 / 100, 2.0)
        assert np.abs(got - ref).max() <= H.TOL_FP32_IMG, (W, Hh)
    cams = [dict(eye=[0, 0, 3], target=[0, 0, 6], up=[0, 1, 0], fovy=0.5)]
    got, ns = _render_gpu(S, net, cams, tf, 16, 16, 1 / 100, 0.99)
    assert ns == 0 and np.all(got == 0)


def test_render_fp32_cfg2_network_sampled_pixels(srn):
    """The config-2 network (32^3 x 16 grid, m = 14, 4 SnakeAlt layers) in
    FP32 at 1024 x 1024, step 1/512: sampled pixels against the oracle."""
    import torch
    S = srn
    p = H.cfg2_params(seed=2)
    net = S.Network(p)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(1)
    W = Hh = 1024
    got, _ = _render_gpu(S, net, cams, tf, W, Hh, 1 / 512, 0.99)
    pix = synth.sample_pixels(1, 1, Hh, W, 300, seed=3)
    ref, mg, _ = oracle.render(oracle.OracleNet(p), cams, H.oracle_tf(tf), W, Hh, 1 / 512, 0.99, pixels=pix,
                               want_margin=True)
    r = H.compare_images(got.reshape(-1, 4)[pix], ref, mg, H.TOL_FP32_IMG, 0.99)
    assert r["ok"], r


@pytest.mark.parametrize("shading", [1, 2, 3])
def test_render_fp32_shading_modes(srn, shading):
    S = srn
    out_dim = 4 if shading == 3 else 1
    p = synth.random_params(R=8, F=8, m=12, layers=3, width=32, out_dim=out_dim, act=synth.ACT_SNAKEALT, seed=4,
                            grid_std=0.5, bias_std=0.2)
    net = S.Network(p)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    got, _ = _render_gpu(S, net, cams, tf, 40, 24, 1 / 64, 2.0, shading=shading, fd_h=1 / 64)
    ref, bound = oracle.render_shade_bound(oracle.OracleNet(p), cams, H.oracle_tf(tf), 40, 24, 1 / 64, 2.0, shading,
                                           oracle.PREC_FP32, fd_h=1 / 64)
    # per pixel: the FP32 image bound plus what the FP32 gradient error bound
    # moves through the shading formula
    r = H.compare_images(got[0], ref[0], None, H.shaded_tol(H.TOL_FP32_IMG, bound[0]), 2.0)
    print(f"fp32 shading {shading}: max error {r['max_strict']:.2e}, worst error / bound {r['worst_ratio']:.2f}")
    assert r["ok"], r


def test_render_fp32_time_interpolation(srn):
    S = srn
    p = synth.random_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SNAKEALT, seed=5, grid_std=0.5,
                            n_keyframes=3, key_times=[0.0, 4.0, 15.0])
    net = S.Network(p)
    tf = synth.tf_preset(4)
    cams = synth.orbit_cameras(2)
    times = [0.0, 2.5, 4.0, 9.0, 15.0, 20.0]
    got, _ = _render_gpu(S, net, cams, tf, 24, 16, 1 / 64, 2.0, times=times)
    ref, _, _ = oracle.render(oracle.OracleNet(p), cams, H.oracle_tf(tf), 24, 16, 1 / 64, 2.0, times=times)
    assert np.abs(got - ref).max() <= H.TOL_FP32_IMG


@pytest.mark.parametrize("shading", [0, 2])
def test_dvr_dense_parity(srn, shading):
    import torch
    S = srn
    vol = synth.blobs_volume(64, 8, seed=6)
    tf = synth.tf_preset(4)
    cams = synth.orbit_cameras(3)
    out = torch.zeros((3, 50, 70, 4), device="cuda")
    ns = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.srn_dvr_dense(vol.cuda(), cams, tf, S.render_desc(70, 50, 1 / 128, 0.99, shading), out, samples=ns)
    torch.cuda.synchronize()
    ref, mg, ns_ref = oracle.dvr_dense(vol.numpy(), cams, H.oracle_tf(tf), 70, 50, 1 / 128, 0.99, shading=shading,
                                       want_margin=True)
    tol = H.TOL_FP32_IMG
    if shading:
        _, bound = oracle.dvr_dense_shade_bound(vol.numpy(), cams, H.oracle_tf(tf), 70, 50, 1 / 128, 0.99,
                                                H.dense_sample_error(vol.numpy()))
        tol = H.shaded_tol(H.TOL_FP32_IMG, bound)
    r = H.compare_images(out.cpu().numpy(), ref, mg, tol, 0.99)
    assert r["ok"], r
    assert abs(int(ns.item()) - ns_ref) <= 0.001 * ns_ref


@pytest.mark.parametrize("dims", [(40, 29, 23), (37, 29, 23)])
@pytest.mark.parametrize("shading", [0, 2])
def test_dvr_dense_anisotropic(srn, dims, shading):
    """Anisotropic volumes: nx a multiple of 4 (rows read by aligned 16-byte
    loads) and nx = 37 (rows read by 4-byte loads); per-axis FD steps."""
    import torch
    S = srn
    nx, ny, nz = dims
    vol = np.ascontiguousarray(synth.blobs_volume(40, 6, seed=9).numpy()[:nz, :ny, :nx])
    tf = synth.tf_preset(4)
    cams = synth.orbit_cameras(3)
    out = torch.zeros((3, 36, 44, 4), device="cuda")
    S.srn_dvr_dense(torch.tensor(vol, device="cuda"), cams, tf, S.render_desc(44, 36, 1 / 96, 0.99, shading), out)
    torch.cuda.synchronize()
    ref, mg, _ = oracle.dvr_dense(vol, cams, H.oracle_tf(tf), 44, 36, 1 / 96, 0.99, shading=shading, want_margin=True)
    tol = H.TOL_FP32_IMG
    if shading:
        _, bound = oracle.dvr_dense_shade_bound(vol, cams, H.oracle_tf(tf), 44, 36, 1 / 96, 0.99,
                                                H.dense_sample_error(vol))
        tol = H.shaded_tol(H.TOL_FP32_IMG, bound)
    r = H.compare_images(out.cpu().numpy(), ref, mg, tol, 0.99)
    assert r["ok"], r


def test_dvr_dense_full_size_sampled(srn):
    """Config 2 dense volume size (256^3) at 1024 x 1024: sampled pixels."""
    import torch
    S = srn
    vol = synth.noise_volume(256, seed=7, device="cuda")
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(1)
    out = torch.zeros((1, 1024, 1024, 4), device="cuda")
    S.srn_dvr_dense(vol, cams, tf, S.render_desc(1024, 1024, 1 / 512, 0.99), out)
    torch.cuda.synchronize()
    pix = synth.sample_pixels(1, 1, 1024, 1024, 400, seed=8)
    ref, mg, _ = oracle.dvr_dense(vol.cpu().numpy(), cams, H.oracle_tf(tf), 1024, 1024, 1 / 512, 0.99, pixels=pix,
                                  want_margin=True)
    r = H.compare_images(out.reshape(-1, 4).cpu().numpy()[pix], ref, mg, H.TOL_FP32_IMG, 0.99)
    assert r["ok"], r


@pytest.mark.parametrize("which", ["cfg1", "cfg2", "head"])
def test_eval_and_density_grad(srn, which):
    import torch
    S = srn
    if which == "cfg1":
        p = H.cfg1_params(seed=9)
    elif which == "cfg2":
        p = H.cfg2_params(seed=10)
    else:
        p = H.cfg2_params(seed=11, out_dim=4)
    net = S.Network(p)
    rng = np.random.default_rng(12)
    n = 1000
    pts = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    pts[:4] = [[0, 0, 0], [1, 1, 1], [0.5, 1.0, 0.0], [1e-7, 0.999999, 0.5]]  # faces and corners
    pt = torch.tensor(pts, device="cuda")
    D = net.out_dim
    out = torch.zeros((n, D), device="cuda")
    S.srn_eval(net.ctx, pt, out)
    rho = torch.zeros(n, device="cuda")
    grad = torch.zeros((n, 3), device="cuda")
    S.srn_density_grad(net.ctx, pt, rho, grad)
    torch.cuda.synchronize()
    on = oracle.OracleNet(p)
    ref = oracle.net_forward(on, pts)
    assert H.rel_density_err(out.cpu().numpy(), ref).max() <= H.TOL_FP32_RHO
    r2, g2 = oracle.net_input_grad(on, pts)
    assert H.rel_density_err(rho.cpu().numpy(), r2).max() <= H.TOL_FP32_RHO
    # per component: the first-order bound of the FP32 path's gradient error
    B = oracle.error_bounds(on, pts, oracle.PREC_FP32)[1]
    ratio = np.abs(grad.cpu().numpy() - g2) / B
    print(f"fp32 adjoint gradient {which}: worst error / bound {ratio.max():.2f}")
    assert ratio.max() <= 1.0


def test_eval_empty_and_time(srn):
    import torch
    S = srn
    p = synth.random_params(R=6, F=8, m=6, layers=3, width=32, act=synth.ACT_SINE, seed=13, grid_std=0.5,
                            n_keyframes=2, key_times=[0.0, 1.0])
    net = S.Network(p)
    S.srn_eval(net.ctx, torch.zeros((0, 3), device="cuda"), torch.zeros((0, 1), device="cuda"))
    pts = np.random.default_rng(14).uniform(0, 1, (64, 3)).astype(np.float32)
    out = torch.zeros((64, 1), device="cuda")
    S.srn_eval(net.ctx, torch.tensor(pts, device="cuda"), out, time=0.3)
    torch.cuda.synchronize()
    ref = oracle.net_forward(oracle.OracleNet(p), pts, 0.3)
    assert H.rel_density_err(out.cpu().numpy(), ref).max() <= H.TOL_FP32_RHO


def test_image_mse(srn):
    import torch
    S = srn
    a = torch.rand((33, 17, 4), device="cuda")
    b = a.clone()
    b[..., :3] += 0.01
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.srn_image_mse(a, b, out)
    torch.cuda.synchronize()
    ref = 10 ** (-oracle.psnr(a.cpu().numpy(), b.cpu().numpy()) / 10)
    assert abs(out.item() - ref) <= 1e-9


@pytest.mark.parametrize("h,w", [(23, 37), (11, 11), (10, 40), (64, 75), (1, 1)])
def test_image_ssim(srn, h, w):
    """SSIM against the FP64 oracle on ragged tiles, a single window, no
    window (1 by convention); identical images give exactly 1; two calls agree
    bit for bit."""
    import torch
    S = srn
    g = torch.Generator(device="cuda").manual_seed(h * 1000 + w)
    a = torch.rand((h, w, 4), device="cuda", generator=g)
    b = (a + 0.2 * torch.rand((h, w, 4), device="cuda", generator=g)).clamp(0, 1)
    b[: h // 2] = a[: h // 2]  # half the image identical: SSIM near 1 there
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    S.srn_image_ssim(a, b, out[0:1])
    S.srn_image_ssim(a, b, out[1:2])
    S.srn_image_ssim(a, a, out[2:3])
    torch.cuda.synchronize()
    ref = oracle.ssim(a.cpu().numpy(), b.cpu().numpy())
    assert abs(out[0].item() - ref) <= 1e-12, (out[0].item(), ref)
    assert out[0].item() == out[1].item() and out[2].item() == 1.0


def test_image_ssim_constant_images(srn):
    """Two constant images: (2 mu_a mu_b + C1) / (mu_a^2 + mu_b^2 + C1)."""
    import torch
    S = srn
    a = torch.full((40, 70, 4), 0.3, device="cuda")
    b = torch.full((40, 70, 4), 0.6, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.srn_image_ssim(a, b, out)
    torch.cuda.synchronize()
    C1 = 0.01 ** 2
    ma, mb = float(np.float32(0.3)), float(np.float32(0.6))
    assert abs(out.item() - (2 * ma * mb + C1) / (ma * ma + mb * mb + C1)) <= 1e-12


@pytest.mark.parametrize("n", [0, 1, 1000, 1025, 4194307])
def test_mse_reductions(srn, n):
    """Density and image MSE against FP64 numpy: empty input, fewer values
    than partial sums, a ragged last range, 4 M values; two calls agree bit
    for bit."""
    import torch
    S = srn
    g = torch.Generator(device="cuda").manual_seed(n)
    a = torch.rand(4 * n, device="cuda", generator=g)
    b = torch.rand(4 * n, device="cuda", generator=g)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    an, bn = a.double().cpu().numpy(), b.double().cpu().numpy()
    S.srn_density_mse(a, b, out[0:1])
    S.srn_density_mse(a, b, out[1:2])
    torch.cuda.synchronize()
    ref = float(np.mean((an - bn) ** 2)) if n else 0.0
    assert abs(out[0].item() - ref) <= 1e-12 * max(ref, 1.0) and out[0].item() == out[1].item()
    S.srn_image_mse(a.view(-1, 4), b.view(-1, 4), out[0:1])
    torch.cuda.synchronize()
    d = (an - bn).reshape(-1, 4)[:, :3]
    ref = float(np.mean(d ** 2)) if n else 0.0
    assert abs(out[0].item() - ref) <= 1e-12 * max(ref, 1.0)
