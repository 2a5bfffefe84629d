"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point that include/srn.h declares, and rejects invalid arguments
before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "srn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(srn_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_01579_gb300 import build
    build.build()
    from paper_2112_01579_gb300 import srn
    return srn


def test_header_declares_the_boundary():
    d = _declared()
    for name in ["srn_create", "srn_destroy", "srn_render", "srn_dvr_dense", "srn_eval", "srn_density_grad",
                 "srn_backward", "srn_fit_step", "srn_sync_status", "srn_last_error"]:
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) <= set(lib.EXPORTED) | set(_declared())
    assert "sm_103a" in lib.srn_version()


def test_create_rejects_bad_configs_without_a_device(lib):
    L = lib.lib()
    h = C.c_void_p()
    p = lib.srn_params()
    assert L.srn_create(None, C.byref(p), C.byref(h)) == lib.SRN_ERR_INVALID_ARG
    cfg = lib.srn_config()
    cfg.grid_res, cfg.feat, cfg.n_fourier, cfg.layers, cfg.width, cfg.out_dim = 8, 8, 12, 2, 32, 1
    cfg.n_keyframes = 1
    bad = [("grid_res", 1, lib.SRN_ERR_INVALID_ARG), ("feat", 6, lib.SRN_ERR_INVALID_ARG),
           ("layers", 1, lib.SRN_ERR_INVALID_ARG), ("out_dim", 2, lib.SRN_ERR_INVALID_ARG),
           ("activation", 7, lib.SRN_ERR_INVALID_ARG), ("width", 40, lib.SRN_ERR_UNSUPPORTED),
           ("n_keyframes", 0, lib.SRN_ERR_INVALID_ARG), ("layers", 12, lib.SRN_ERR_UNSUPPORTED),
           ("precision", lib.SRN_PREC_BF16, lib.SRN_ERR_UNSUPPORTED), ("precision", 3, lib.SRN_ERR_INVALID_ARG)]
    for field, val, st in bad:
        c2 = lib.srn_config.from_buffer_copy(cfg)
        setattr(c2, field, val)
        assert L.srn_create(C.byref(c2), C.byref(p), C.byref(h)) == st, field
        assert lib.srn_last_error() != ""
    # valid config, missing parameter pointers
    assert L.srn_create(C.byref(cfg), C.byref(p), C.byref(h)) == lib.SRN_ERR_INVALID_ARG
    # non-increasing keyframe times
    c3 = lib.srn_config.from_buffer_copy(cfg)
    c3.n_keyframes = 3
    c3.key_times[0], c3.key_times[1], c3.key_times[2] = 0.0, 2.0, 1.0
    assert L.srn_create(C.byref(c3), C.byref(p), C.byref(h)) == lib.SRN_ERR_INVALID_ARG


def test_calls_reject_null_contexts_and_bad_batches(lib):
    L = lib.lib()
    desc = lib.render_desc(16, 16, 0.01)
    cams = lib._cams([dict(eye=[0, 0, 2], target=[0, 0, 0], up=[0, 1, 0], fovy=1.0)])
    tf = lib.make_tf(dict(pos=[0, 1], rgba=[[0, 0, 0, 0], [1, 1, 1, 1]], opacity_scale=1.0))
    assert L.srn_render(None, cams, 1, None, 1, C.byref(tf), C.byref(desc), None, None, None) == lib.SRN_ERR_INVALID_ARG
    assert L.srn_eval(None, None, 0, 0.0, None, None) == lib.SRN_ERR_INVALID_ARG
    dims = (C.c_int * 3)(1, 4, 4)
    fake = C.c_void_p(0x10000)
    assert L.srn_dvr_dense(fake, dims, cams, 1, C.byref(tf), C.byref(desc), fake, None, None) == lib.SRN_ERR_INVALID_ARG
    dims = (C.c_int * 3)(4, 4, 4)
    for d in [lib.render_desc(0, 16, 0.01), lib.render_desc(16, 16, 0.0), lib.render_desc(16, 16, 0.01, shading=9),
              lib.render_desc(16, 16, 0.01, shading=lib.SRN_SHADE_ADJOINT)]:
        assert L.srn_dvr_dense(fake, dims, cams, 1, C.byref(tf), C.byref(d), fake, None, None) == \
            lib.SRN_ERR_INVALID_ARG
    unsorted = lib.make_tf(dict(pos=[0.5, 0.2], rgba=[[0, 0, 0, 0], [1, 1, 1, 1]], opacity_scale=1.0))
    assert L.srn_dvr_dense(fake, dims, cams, 1, C.byref(unsorted), C.byref(desc), fake, None, None) == \
        lib.SRN_ERR_INVALID_ARG
    degenerate = lib._cams([dict(eye=[0, 0, 2], target=[0, 0, 2], up=[0, 1, 0], fovy=1.0)])
    assert L.srn_dvr_dense(fake, dims, degenerate, 1, C.byref(tf), C.byref(desc), fake, None, None) == \
        lib.SRN_ERR_INVALID_ARG
    misaligned = C.c_void_p(0x10004)
    assert L.srn_dvr_dense(fake, dims, cams, 1, C.byref(tf), C.byref(desc), misaligned, None, None) == \
        lib.SRN_ERR_INVALID_ARG
    assert L.srn_image_mse(fake, fake, -1, fake, None) == lib.SRN_ERR_INVALID_ARG
    assert L.srn_fit_steps(None, fake, dims, 16, 1, 0, 4, 0.0, 1e-2, 5e-3, 0.0, 1.0, fake, None) == \
        lib.SRN_ERR_INVALID_ARG
    for w, h, pa, out in ((0, 4, fake, fake), (4, -1, fake, fake), (4, 4, None, fake), (4, 4, fake, None),
                          (4, 4, misaligned, fake)):
        assert L.srn_image_ssim(pa, fake, w, h, out, None) == lib.SRN_ERR_INVALID_ARG
