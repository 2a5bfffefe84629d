"""Transfer-function and batch edge cases through the C ABI against the FP64
oracle: the maximum number of control points (32), two points with flat
extension outside them, a zero-width segment (duplicate position), and the
maximum number of views (64) in one call; FP32 and FP16 renders and dense
DVR.  The transfer functions are continuous with slopes like the presets'
(a jump in the TF would let an error within the bound flip a colour, where
several results are correct)."""
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


def _tf(kind):
    if kind == "max32":
        rng = np.random.default_rng(5)
        pos = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0.02, 0.98, 30)])).astype(np.float32)
        ph = rng.uniform(0, 2 * math.pi, 4)
        rgba = np.stack([0.5 + 0.4 * np.sin(2 * math.pi * 0.6 * pos + ph[c]) for c in range(3)] +
                        [0.3 + 0.25 * np.sin(2 * math.pi * 0.5 * pos + ph[3])], axis=1).astype(np.float32)
    elif kind == "two":
        pos = np.asarray([0.3, 0.7], np.float32)
        rgba = np.asarray([[0.1, 0.2, 0.9, 0.02], [1.0, 0.6, 0.2, 0.6]], np.float32)
    elif kind == "tie":
        pos = np.asarray([0.0, 0.45, 0.45, 0.7, 1.0], np.float32)
        rgba = np.asarray([[0.0, 0.0, 0.0, 0.0], [0.3, 0.6, 1.0, 0.2], [0.3, 0.6, 1.0, 0.2], [1.0, 0.5, 0.2, 0.5],
                           [1.0, 1.0, 1.0, 0.9]], np.float32)
    else:
        raise ValueError(kind)
    assert len(pos) <= 32
    return dict(pos=pos, rgba=rgba, opacity_scale=20.0)


def _render(S, net, cams, tf, W, Hh, step, et):
    import torch
    out = torch.full((1, len(cams), Hh, W, 4), -1.0, device="cuda")
    S.srn_render(net.ctx, cams, tf, S.render_desc(W, Hh, step, et), out)
    torch.cuda.synchronize()
    st, msg = S.srn_sync_status(net.ctx)
    assert st == 0, msg
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", ["max32", "two", "tie"])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_transfer_function_edge_cases(srn, kind, precision):
    S = srn
    p = H.cfg2_params(seed=90, R=16)
    if precision == "fp16":
        p = synth.to_half_exact(p)
        net, tol = S.Network(p, precision=S.SRN_PREC_FP16), H.TOL_FP16_IMG
    else:
        net, tol = S.Network(p), H.TOL_FP32_IMG
    tf = _tf(kind)
    cams = synth.orbit_cameras(2)
    for et in (2.0, 0.99):
        got = _render(S, net, cams, tf, 40, 30, 1 / 96, et)
        ref, mg, _ = oracle.render(oracle.OracleNet(p), cams, H.oracle_tf(tf), 40, 30, 1 / 96, et, want_margin=True)
        assert np.all(got >= 0)
        r = H.compare_images(got[0], ref[0], mg[0], tol, et)
        assert r["ok"], (kind, precision, et, r)
    net.close()


@pytest.mark.parametrize("kind", ["max32", "two", "tie"])
def test_transfer_function_edge_cases_dense(srn, kind):
    import torch
    S = srn
    vol = synth.blobs_volume(40, 6, seed=91)
    tf = _tf(kind)
    cams = synth.orbit_cameras(2)
    out = torch.zeros((2, 30, 40, 4), device="cuda")
    S.srn_dvr_dense(vol.cuda(), cams, tf, S.render_desc(40, 30, 1 / 96, 0.99), out)
    torch.cuda.synchronize()
    ref, mg, _ = oracle.dvr_dense(vol.numpy(), cams, H.oracle_tf(tf), 40, 30, 1 / 96, 0.99, want_margin=True)
    r = H.compare_images(out.cpu().numpy(), ref, mg, H.TOL_FP32_IMG, 0.99)
    assert r["ok"], (kind, r)


def test_maximum_views_in_one_call(srn):
    """64 views (the limit) in one FP16 render and one dense call; 65 is
    rejected before any launch."""
    import torch
    S = srn
    p = synth.to_half_exact(H.cfg2_params(seed=92, R=16))
    net = S.Network(p, precision=S.SRN_PREC_FP16)
    tf = synth.tf_preset(8)
    cams = [dict(eye=[math.cos(a) * math.cos(e), math.sin(e), math.sin(a) * math.cos(e)], target=[0, 0, 0],
                 up=[0, 1, 0], fovy=math.radians(60))
            for a, e in zip(np.linspace(0, 2 * math.pi, 64, endpoint=False), np.linspace(-1.2, 1.2, 64))]
    got = _render(S, net, cams, tf, 12, 10, 1 / 64, 0.99)
    ref, mg, _ = oracle.render(oracle.OracleNet(p), cams, H.oracle_tf(tf), 12, 10, 1 / 64, 0.99, want_margin=True)
    r = H.compare_images(got[0], ref[0], mg[0], H.TOL_FP16_IMG, 0.99)
    assert r["ok"], r
    vol = synth.blobs_volume(24, 5, seed=93)
    dense = torch.zeros((64, 10, 12, 4), device="cuda")
    S.srn_dvr_dense(vol.cuda(), cams, tf, S.render_desc(12, 10, 1 / 64, 0.99), dense)
    torch.cuda.synchronize()
    dref, dmg, _ = oracle.dvr_dense(vol.numpy(), cams, H.oracle_tf(tf), 12, 10, 1 / 64, 0.99, want_margin=True)
    r = H.compare_images(dense.cpu().numpy(), dref, dmg, H.TOL_FP32_IMG, 0.99)
    assert r["ok"], r
    too_many = torch.zeros((65, 10, 12, 4), device="cuda")
    with pytest.raises(Exception):
        S.srn_render(net.ctx, cams + cams[:1], tf, S.render_desc(12, 10, 1 / 64, 0.99), too_many)
    net.close()
