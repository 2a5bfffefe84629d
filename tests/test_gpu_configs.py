"""Parity at the full sizes of the shaded and time-varying workloads (sampled
pixels against the oracle, same launch configuration as a full render), and
the learned-vs-plain comparison of Section 6.2."""
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


def _render(S, net, cams, tf, W, Hh, step, et, shading=0, fd_h=0.0, times=None):
    import torch
    T = 1 if times is None else len(times)
    out = torch.full((T, len(cams), Hh, W, 4), -1.0, device="cuda")
    S.srn_render(net.ctx, cams, tf, S.render_desc(W, Hh, step, et, shading, fd_h), out, times=times)
    torch.cuda.synchronize()
    assert S.srn_sync_status(net.ctx)[0] == 0
    return out


@pytest.mark.parametrize("shading,precision", [(1, 0), (1, 1), (2, 1), (3, 1)])
def test_shaded_workload_full_size(srn, shading, precision):
    """64^3 x 16 latent grid, 4 SnakeAlt layers of width 32, 1024^2 at step
    1/1024, headlight Blinn-Phong from the adjoint (FP32 or FP16 path), central
    differences with a one-voxel step of the 512^3 volume (FP16 path) or the
    4-output head (FP16 path)."""
    S = srn
    p = H.cfg2_params(seed=80, R=64, out_dim=4 if shading == 3 else 1)
    q = synth.to_half_exact(p) if precision == 1 else p
    net = S.Network(q, precision=precision)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(1)
    out = _render(S, net, cams, tf, 1024, 1024, 1 / 1024, 0.99, shading=shading, fd_h=1 / 511)
    pix = synth.sample_pixels(1, 1, 1024, 1024, 96, seed=81)
    on = oracle.OracleNet(q)
    ref, mg, _ = oracle.render(on, cams, H.oracle_tf(tf), 1024, 1024, 1 / 1024, 0.99, shading=shading, fd_h=1 / 511,
                               pixels=pix, want_margin=True)
    _, bound = oracle.render_shade_bound(on, cams, H.oracle_tf(tf), 1024, 1024, 1 / 1024, 0.99, shading,
                                         oracle.PREC_FP32 if precision == 0 else oracle.PREC_FP16, fd_h=1 / 511,
                                         pixels=pix)
    got = out.reshape(-1, 4).cpu().numpy()[pix]
    img_tol = H.TOL_FP32_IMG if precision == 0 else H.TOL_FP16_IMG
    r = H.compare_images(got, ref, mg, H.shaded_tol(img_tol, bound), 0.99)
    print(f"shaded workload {shading}/{precision}: max error {r['max_strict']:.2e}, worst error / bound "
          f"{r['worst_ratio']:.2f}")
    assert r["ok"], r


def test_shaded_dense_dvr_512(srn):
    """Dense DVR of the 512^3 anisotropic-blob volume with one-voxel central
    differences, 1024^2 at step 1/1024."""
    import torch
    S = srn
    vol = synth.aniso_blobs_volume(512, 64, seed=82, device="cuda")
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(1)
    out = torch.zeros((1, 1024, 1024, 4), device="cuda")
    S.srn_dvr_dense(vol, cams, tf, S.render_desc(1024, 1024, 1 / 1024, 0.99, 2), out)
    torch.cuda.synchronize()
    pix = synth.sample_pixels(1, 1, 1024, 1024, 96, seed=83)
    vol_np = vol.cpu().numpy()
    ref, mg, _ = oracle.dvr_dense(vol_np, cams, H.oracle_tf(tf), 1024, 1024, 1 / 1024, 0.99, shading=2,
                                  pixels=pix, want_margin=True)
    _, bound = oracle.dvr_dense_shade_bound(vol_np, cams, H.oracle_tf(tf), 1024, 1024, 1 / 1024, 0.99,
                                            H.dense_sample_error(vol_np), pixels=pix)
    r = H.compare_images(out.reshape(-1, 4).cpu().numpy()[pix], ref, mg, H.shaded_tol(H.TOL_FP32_IMG, bound), 0.99)
    print(f"shaded dense 512: max error {r['max_strict']:.2e}, worst error / bound {r['worst_ratio']:.2f}")
    assert r["ok"], r


def test_time_batch_full_size(srn):
    """Five 32^3 x 16 keyframe grids (0, 4, 8, 12, 15), 16 times x 4 views at
    1024^2 in one launch, step 1/512."""
    S = srn
    p = H.cfg2_params(seed=84, nkey=5, key_times=[0, 4, 8, 12, 15])
    q = synth.to_half_exact(p)
    net = S.Network(q, precision=S.SRN_PREC_FP16)
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(4)
    times = list(range(16))
    out = _render(S, net, cams, tf, 1024, 1024, 1 / 512, 0.99, times=times)
    assert float(out.min()) >= 0.0  # every pixel of the batch written
    pix = synth.sample_pixels(16, 4, 1024, 1024, 160, seed=85)
    ref, mg, _ = oracle.render(oracle.OracleNet(q), cams, H.oracle_tf(tf), 1024, 1024, 1 / 512, 0.99, times=times,
                               pixels=pix, want_margin=True)
    r = H.compare_images(out.reshape(-1, 4).cpu().numpy()[pix], ref, mg, H.TOL_FP16_IMG, 0.99)
    assert r["ok"], r


def test_learned_network_beats_equal_memory_lowpass_grid(srn):
    """Section 6.2: at equal memory the fitted fV-SRN (16^3 x 16 latent grid)
    reconstructs a fine-detail volume better than the low-pass density grid
    of the same size (M = round(cbrt(16^3 * 16)) = 40), in density PSNR and
    in rendered-image PSNR against dense DVR of the full volume."""
    import torch
    S = srn
    n = 128
    vol = synth.noise_volume(n, seed=86, device="cuda").contiguous()
    p = synth.init_params(R=16, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=87)
    net = S.Network(p, precision=S.SRN_PREC_FP16, max_fit_points=1 << 16, adam=True)
    loss = torch.zeros(1, device="cuda")
    for s in range(800):
        S.srn_fit_step(net.ctx, vol, 1 << 16, 5, s, loss)
    S.srn_sync_half(net.ctx)
    x = torch.linspace(0, 1, n, device="cuda")
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    pts = torch.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1).contiguous()
    rho = torch.empty((pts.shape[0], 1), device="cuda")
    S.srn_eval(net.ctx, pts, rho)
    mse = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.srn_density_mse(rho[:, 0].contiguous(), vol.reshape(-1), mse)
    torch.cuda.synchronize()
    psnr_net = 10 * math.log10(1 / mse.item())
    M = round((16 ** 3 * 16) ** (1 / 3))
    assert M == 40
    tmp = torch.empty(2 * vol.numel(), device="cuda")
    grid = torch.empty((M, M, M), device="cuda")
    S.srn_lowpass_resample(vol, M, tmp, grid)
    back = torch.empty_like(vol)
    S.srn_resample(grid, back)
    S.srn_density_mse(back, vol, mse)
    torch.cuda.synchronize()
    psnr_lp = 10 * math.log10(1 / mse.item())
    tf = synth.tf_preset(8)
    cams = synth.orbit_cameras(2)
    desc = S.render_desc(256, 256, 1 / 256, 0.99)
    img = torch.zeros((1, 2, 256, 256, 4), device="cuda")
    ref = torch.zeros((2, 256, 256, 4), device="cuda")
    lpi = torch.zeros((2, 256, 256, 4), device="cuda")
    S.srn_render(net.ctx, cams, tf, desc, img)
    S.srn_dvr_dense(vol, cams, tf, desc, ref)
    S.srn_dvr_dense(grid, cams, tf, desc, lpi)
    S.srn_image_mse(img[0].contiguous(), ref, mse)
    torch.cuda.synchronize()
    img_net = 10 * math.log10(1 / mse.item())
    S.srn_image_mse(lpi, ref, mse)
    torch.cuda.synchronize()
    img_lp = 10 * math.log10(1 / mse.item())
    print(f"density PSNR fV-SRN {psnr_net:.2f} dB vs low-pass {psnr_lp:.2f} dB; "
          f"image PSNR {img_net:.2f} vs {img_lp:.2f} dB")
    assert psnr_net > psnr_lp
    assert img_net > img_lp
