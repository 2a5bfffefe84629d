"""FP64 CPU oracle for the fV-SRN render / fit path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_2112_01579_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``srn_oracle.c`` (plain C, double precision, each
function citing the paper's section / equation it restates).  This module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

ACT_SINE, ACT_SNAKEALT = 0, 1
SHADE_NONE, SHADE_ADJOINT, SHADE_FD, SHADE_HEAD = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Net(C.Structure):
    _fields_ = [("R", C.c_int), ("F", C.c_int), ("m", C.c_int), ("l", C.c_int), ("c", C.c_int),
                ("D", C.c_int), ("act", C.c_int), ("nkey", C.c_int), ("time_input", C.c_int),
                ("key_times", C.POINTER(C.c_double)), ("grid", C.POINTER(C.c_double)),
                ("fourier", C.POINTER(C.c_double)), ("W", C.POINTER(C.c_double)),
                ("b", C.POINTER(C.c_double))]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
                ("fovy", C.c_double)]


class TF(C.Structure):
    _fields_ = [("n", C.c_int), ("pos", C.POINTER(C.c_double)), ("rgba", C.POINTER(C.c_double)),
                ("opacity_scale", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L = _lib
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.orc_sample_point.argtypes = [C.c_uint64, C.c_int, C.c_int, dp]
            L.orc_trilinear.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
            L.orc_trilinear_grad.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
            L.orc_volume_fd_grad.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, dp]
            L.orc_net_check.argtypes = [C.POINTER(Net)]
            L.orc_net_forward.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_double, dp]
            L.orc_net_backward.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_double, dp, dp, dp, dp]
            L.orc_net_input_grad.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_double, dp, dp]
            L.orc_net_input_vjp.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_double, dp, dp]
            L.orc_tf_eval.argtypes = [C.POINTER(TF), C.c_double, dp]
            L.orc_camera_ray.argtypes = [C.POINTER(Camera), C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
            L.orc_box_intersect.argtypes = [dp, dp, dp, dp]
            L.orc_render.argtypes = [C.POINTER(Net), C.POINTER(Camera), C.c_int, dp, C.c_int, C.POINTER(TF),
                                     C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                     C.POINTER(C.c_longlong), C.c_longlong, dp, dp, C.POINTER(C.c_longlong)]
            L.orc_dvr_dense.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.POINTER(Camera), C.c_int, C.POINTER(TF),
                                        C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                        C.POINTER(C.c_longlong), C.c_longlong, dp, dp, C.POINTER(C.c_longlong)]
            u64p = C.POINTER(C.c_uint64)
            L.orc_fit_loss_grad.restype = C.c_double
            L.orc_fit_loss_grad.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                            C.c_int, C.c_double, C.c_double, C.c_double, dp, dp, dp, u64p, C.c_int]
            L.orc_error_bounds.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_double, dp, dp, dp]
            L.orc_render_shade_bound.argtypes = [C.POINTER(Net), C.POINTER(Camera), C.c_int, dp, C.c_int,
                                                 C.POINTER(TF), C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                                 C.c_double, C.POINTER(C.c_longlong), C.c_longlong, dp, dp, dp]
            L.orc_dvr_dense_shade_bound.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.POINTER(Camera), C.c_int,
                                                    C.POINTER(TF), C.c_int, C.c_int, C.c_double, C.c_double,
                                                    C.POINTER(C.c_longlong), C.c_longlong, dp, dp, dp]
            L.orc_fit_residuals.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                            C.c_int, C.c_double, u64p, C.c_int, dp, dp]
            L.orc_adam.argtypes = [dp, dp, dp, dp, C.c_size_t, C.c_double, C.c_int, C.c_double, C.c_double,
                                   C.c_double]
            L.orc_fit_step.restype = C.c_double
            L.orc_fit_step.argtypes = [C.POINTER(Net), dp, dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                       C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, dp,
                                       C.POINTER(C.c_int), u64p, C.c_int]
            L.orc_error_grid.argtypes = [C.POINTER(Net), dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                         C.c_double, dp]
            L.orc_adaptive_cdf.restype = C.c_int
            L.orc_adaptive_cdf.argtypes = [C.POINTER(C.c_float), C.c_int, u64p]
            L.orc_adaptive_point.argtypes = [u64p, C.c_int, C.c_uint64, C.c_int, C.c_int, C.c_int, dp]
            L.orc_lowpass_resample.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, dp]
            L.orc_psnr.restype = C.c_double
            L.orc_psnr.argtypes = [dp, dp, C.c_longlong]
            L.orc_ssim.restype = C.c_double
            L.orc_ssim.argtypes = [dp, dp, C.c_int, C.c_int]
        return _lib


def _d(a):
    """Contiguous float64 copy (exact widening of FP32 / FP16 values)."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleNet:
    """FP64 copy of an fV-SRN parameter set, kept alive for the C calls.

    ``params`` is a dict with ``grid`` ([nkey, R, R, R, F]), ``fourier``
    ([m, 3]), ``weights`` (list of [d_out, d_in]) and ``biases`` (list), plus
    the config fields ``act`` and optional ``key_times``.
    """

    def __init__(self, params: dict):
        self.grid = _d(params["grid"]).reshape(-1)
        g = np.asarray(params["grid"])
        nkey, R = g.shape[0], g.shape[1]
        F = g.shape[4]
        self.fourier = _d(params["fourier"]).reshape(-1)
        m = len(self.fourier) // 3
        Ws = [np.asarray(w) for w in params["weights"]]
        self.W = np.concatenate([_d(w).reshape(-1) for w in Ws])
        self.b = np.concatenate([_d(b).reshape(-1) for b in params["biases"]])
        self.key_times = _d32(params.get("key_times", np.zeros(max(nkey, 1)))).reshape(-1)
        c = Ws[0].shape[0] if len(Ws) > 1 else 0
        D = Ws[-1].shape[0]
        ti = int(params.get("time_input", 0))
        self.dims = dict(R=R, F=F, m=m, l=len(Ws), c=c, D=D, act=int(params["act"]), nkey=nkey, time_input=ti)
        self.layer_shapes = [w.shape for w in Ws]
        self.s = Net(R, F, m, len(Ws), c, D, int(params["act"]), nkey, ti, _p(self.key_times), _p(self.grid),
                     _p(self.fourier), _p(self.W), _p(self.b))
        if lib().orc_net_check(C.byref(self.s)) != 0:
            raise ValueError("network outside the oracle's limits")

    def unpack_W(self, flat):
        out, o = [], 0
        for s in self.layer_shapes:
            n = s[0] * s[1]
            out.append(np.asarray(flat[o:o + n]).reshape(s))
            o += n
        return out

    def unpack_b(self, flat):
        out, o = [], 0
        for s in self.layer_shapes:
            out.append(np.asarray(flat[o:o + s[0]]))
            o += s[0]
        return out


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def sample_points(seed: int, step: int, n: int) -> np.ndarray:
    out = np.zeros((n, 3))
    for j in range(n):
        lib().orc_sample_point(seed, step, j, _p(out[j]))
    return out


def trilinear(vol, p):
    """vol [nz, ny, nx] or [nz, ny, nx, C]; p [3] in [0,1]^3."""
    v = _d(vol)
    if v.ndim == 3:
        v = v[..., None]
    nz, ny, nx, Cc = v.shape
    out = np.zeros(Cc)
    lib().orc_trilinear(_p(v), nx, ny, nz, Cc, _p(_d(p)), _p(out))
    return out


def trilinear_grad(vol, p):
    v = _d(vol)
    if v.ndim == 3:
        v = v[..., None]
    nz, ny, nx, Cc = v.shape
    out = np.zeros((Cc, 3))
    lib().orc_trilinear_grad(_p(v), nx, ny, nz, Cc, _p(_d(p)), _p(out))
    return out


def volume_fd_grad(vol, p):
    """One-voxel central differences of the trilinear volume [nz, ny, nx] at
    p [3] in [0,1]^3 (the dense-grid shading gradient and the head's
    targets)."""
    v = _d(vol)
    nz, ny, nx = v.shape
    g = np.zeros(3)
    lib().orc_volume_fd_grad(_p(v), nx, ny, nz, _p(_d(p)), _p(g))
    return g


def net_forward(net: OracleNet, pts, t: float = 0.0) -> np.ndarray:
    P = _d(pts).reshape(-1, 3)
    out = np.zeros((len(P), net.dims["D"]))
    lib().orc_net_forward(C.byref(net.s), _p(P), len(P), _f32(t), _p(out))
    return out


def net_backward(net: OracleNet, pts, dout, t: float = 0.0):
    """Gradients of sum_j <dout_j, net(p_j)> w.r.t. (W list, b list, grid)."""
    P = _d(pts).reshape(-1, 3)
    G = _d(dout).reshape(len(P), net.dims["D"])
    dW = np.zeros_like(net.W)
    db = np.zeros_like(net.b)
    dg = np.zeros_like(net.grid)
    lib().orc_net_backward(C.byref(net.s), _p(P), len(P), _f32(t), _p(G), _p(dW), _p(db), _p(dg))
    return net.unpack_W(dW), net.unpack_b(db), dg


def net_input_grad(net: OracleNet, pts, t: float = 0.0):
    P = _d(pts).reshape(-1, 3)
    rho = np.zeros(len(P))
    g = np.zeros((len(P), 3))
    lib().orc_net_input_grad(C.byref(net.s), _p(P), len(P), _f32(t), _p(rho), _p(g))
    return rho, g


def net_input_vjp(net: OracleNet, pts, dout, t: float = 0.0):
    """grad [n, 3] = sum_d dout[:, d] d out_d / d p."""
    P = _d(pts).reshape(-1, 3)
    G = _d(dout).reshape(len(P), net.dims["D"])
    g = np.zeros((len(P), 3))
    lib().orc_net_input_vjp(C.byref(net.s), _p(P), len(P), _f32(t), _p(G), _p(g))
    return g


def _f32(x):
    """The FP32 value the C ABI receives for a scalar parameter (camera,
    transfer function, step, threshold, time): the oracle is given the same
    value, widened exactly."""
    return float(np.float32(x))


def _d32(a):
    return np.ascontiguousarray(np.asarray(a, np.float32).astype(np.float64))


class OracleTF:
    def __init__(self, pos, rgba, opacity_scale):
        self.pos = _d32(pos).reshape(-1)
        self.rgba = _d32(rgba).reshape(-1)
        self.s = TF(len(self.pos), _p(self.pos), _p(self.rgba), _f32(opacity_scale))


def tf_eval(tf: OracleTF, rho: float):
    out = np.zeros(4)
    lib().orc_tf_eval(C.byref(tf.s), rho, _p(out))
    return out


def _cams(cams):
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].eye[:] = [_f32(v) for v in c["eye"]]
        arr[i].target[:] = [_f32(v) for v in c["target"]]
        arr[i].up[:] = [_f32(v) for v in c["up"]]
        arr[i].fovy = _f32(c["fovy"])
    return arr


def camera_ray(cam, W, H, px, py):
    o, d = np.zeros(3), np.zeros(3)
    lib().orc_camera_ray(_cams([cam]), W, H, px, py, _p(o), _p(d))
    return o, d


def box_intersect(o, d):
    t0, t1 = C.c_double(), C.c_double()
    hit = lib().orc_box_intersect(_p(_d(o)), _p(_d(d)), C.byref(t0), C.byref(t1))
    return bool(hit), t0.value, t1.value


def _pix(pixels):
    if pixels is None:
        return None, 0, None
    pa = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
    return pa.ctypes.data_as(C.POINTER(C.c_longlong)), len(pa), pa


def render(net: OracleNet, cams, tf: OracleTF, W, H, step, et, shading=SHADE_NONE, fd_h=0.0, times=None,
           pixels=None, want_margin=False):
    """fV-SRN render.  Returns (rgba [n_pix, 4] or [T, V, H, W, 4], margin, samples)."""
    T = 1 if times is None else len(times)
    tarr = None if times is None else _d32(times)
    pp, npix, keep = _pix(pixels)
    total = npix if pixels is not None else T * len(cams) * H * W
    out = np.zeros((total, 4))
    mg = np.zeros(total) if want_margin else None
    ns = C.c_longlong()
    lib().orc_render(C.byref(net.s), _cams(cams), len(cams), _p(tarr) if tarr is not None else None, T,
                     C.byref(tf.s), W, H, _f32(step), _f32(et), shading, _f32(fd_h), pp, npix, _p(out),
                     _p(mg) if mg is not None else None, C.byref(ns))
    if pixels is None:
        out = out.reshape(T, len(cams), H, W, 4)
        if mg is not None:
            mg = mg.reshape(T, len(cams), H, W)
    return out, mg, ns.value


def dvr_dense(vol, cams, tf: OracleTF, W, H, step, et, shading=SHADE_NONE, pixels=None, want_margin=False):
    v = _d(vol)
    nz, ny, nx = v.shape
    pp, npix, keep = _pix(pixels)
    total = npix if pixels is not None else len(cams) * H * W
    out = np.zeros((total, 4))
    mg = np.zeros(total) if want_margin else None
    ns = C.c_longlong()
    lib().orc_dvr_dense(_p(v), nx, ny, nz, _cams(cams), len(cams), C.byref(tf.s), W, H, _f32(step), _f32(et), shading, pp,
                        npix, _p(out), _p(mg) if mg is not None else None, C.byref(ns))
    if pixels is None:
        out = out.reshape(len(cams), H, W, 4)
        if mg is not None:
            mg = mg.reshape(len(cams), H, W)
    return out, mg, ns.value


def _cdf_args(cdf):
    """(pointer, res) of an adaptive distribution from adaptive_cdf, or (None, 0)."""
    if cdf is None:
        return None, 0
    S, res = cdf
    assert S.dtype == np.uint64 and S.flags.c_contiguous and S.size == res ** 3 + 1
    return S.ctypes.data_as(C.POINTER(C.c_uint64)), res


def fit_loss_grad(net: OracleNet, vol, n_points, seed, step, t=0.0, gw=0.0, gs=1.0, cdf=None):
    v = _d(vol)
    nz, ny, nx = v.shape
    dW = np.zeros_like(net.W)
    db = np.zeros_like(net.b)
    dg = np.zeros_like(net.grid)
    cp, cres = _cdf_args(cdf)
    loss = lib().orc_fit_loss_grad(C.byref(net.s), _p(v), nx, ny, nz, n_points, seed, step, _f32(t), _f32(gw), _f32(gs), _p(dW),
                                   _p(db), _p(dg), cp, cres)
    return loss, net.unpack_W(dW), net.unpack_b(db), dg


def fit_residuals(net: OracleNet, vol, n_points, seed, step, t=0.0, cdf=None):
    """(r [n], points [n, 3]): density residuals rho(p_j) - y_j of a fit
    step's points, in FP64."""
    v = _d(vol)
    nz, ny, nx = v.shape
    r = np.zeros(n_points)
    P = np.zeros((n_points, 3))
    cp, cres = _cdf_args(cdf)
    lib().orc_fit_residuals(C.byref(net.s), _p(v), nx, ny, nz, n_points, seed, step, _f32(t), cp, cres, _p(r), _p(P))
    return r, P


def error_grid(net: OracleNet, vol, res, spv, seed, t=0.0):
    """Section 6.2 error grid E [res, res, res] (z, y, x) in float64."""
    v = _d(vol)
    nz, ny, nx = v.shape
    E = np.zeros(res ** 3)
    lib().orc_error_grid(C.byref(net.s), _p(v), nx, ny, nz, res, spv, seed, _f32(t), _p(E))
    return E.reshape(res, res, res)


def adaptive_cdf(E_f32, res):
    """Integer distribution (S, res) from FP32 error values; raises on a
    negative or non-finite entry."""
    e = np.ascontiguousarray(np.asarray(E_f32, np.float32).reshape(-1))
    assert e.size == res ** 3
    S = np.zeros(res ** 3 + 1, np.uint64)
    st = lib().orc_adaptive_cdf(e.ctypes.data_as(C.POINTER(C.c_float)), res, S.ctypes.data_as(C.POINTER(C.c_uint64)))
    if st:
        raise ValueError("error grid has a negative or non-finite entry")
    return S, res


def adaptive_points(cdf, seed, step, n):
    S, res = cdf
    out = np.zeros((n, 3))
    sp = S.ctypes.data_as(C.POINTER(C.c_uint64))
    for j in range(n):
        lib().orc_adaptive_point(sp, res, seed, step, j, n, _p(out[j]))
    return out


def adam(theta, m, v, g, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam on float64 arrays."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg = _d(g)
    lib().orc_adam(_p(theta), _p(m), _p(v), _p(gg), theta.size, lr, step, beta1, beta2, eps)


def fit_step(net: OracleNet, adam_m, adam_v, vol, n_points, seed, step, lr_grid, lr_net, t=0.0, gw=0.0, gs=1.0,
             cdf=None):
    """One fit step on the oracle's FP64 parameters (updated in place).

    Returns (loss, grads [grid | W | b] flat, status)."""
    v = _d(vol)
    nz, ny, nx = v.shape
    grads = np.zeros(net.grid.size + net.W.size + net.b.size)
    st = C.c_int()
    cp, cres = _cdf_args(cdf)
    loss = lib().orc_fit_step(C.byref(net.s), _p(adam_m), _p(adam_v), _p(v), nx, ny, nz, n_points, seed, step,
                              _f32(t), _f32(lr_grid), _f32(lr_net), _f32(gw), _f32(gs), _p(grads), C.byref(st), cp,
                              cres)
    return loss, grads, st.value


def lowpass_resample(vol, M):
    v = _d(vol)
    nz, ny, nx = v.shape
    out = np.zeros((M, M, M))
    lib().orc_lowpass_resample(_p(v), nx, ny, nz, M, _p(out))
    return out


def psnr(a, b):
    A, B = _d(a).reshape(-1, 4), _d(b).reshape(-1, 4)
    return lib().orc_psnr(_p(A), _p(B), len(A))


def ssim(a, b):
    A, B = _d(a), _d(b)
    H, W = A.shape[-3], A.shape[-2]
    return lib().orc_ssim(_p(A.reshape(-1)), _p(B.reshape(-1)), W, H)


# ---------------------------------------------------------------- error bounds
# Precision models of the two kernel paths for the first-order bounds (field
# order of orc_prec: in_rel, in_abs, act_abs, act_rel, acc, dact_abs, bwd_rel,
# jac_rel, vol_abs, lat_w).
#  FP16 tensor-core path: layer-0 inputs computed in FP32 and rounded to FP16
#   (half an FP16 ulp, 2^-11, plus the FP32 features' error, 2^-19 absolute);
#   hidden activations from MUFU sin / cos (absolute error ~2^-21 for
#   |x| <= pi, taken as 2^-20 (1 + |x|)) carried as FP16 hi + lo (2^-22);
#   tensor-core FP32 accumulation (2^-23 per term, K terms); derivatives from
#   MUFU as the activations; adjoint rows as hi + lo (2^-22); Fourier and
#   latent Jacobians recomputed in FP32 with angle doubling (2^-17); the
#   trilinear latent weights rounded to FP16 (2^-11 of sum_k w_k |G_k|).
#  FP32 CUDA-core path: inputs from compensated FP32 sin / cos and an FP32
#   trilinear (2^-21 relative, 2^-23 absolute); accurate sinf / sincosf
#   (2^-22); FMA chains (2^-24 per term); Jacobians 2^-21.
PREC_FP16 = (2.0 ** -11, 2.0 ** -19, 2.0 ** -19, 2.0 ** -22, 2.0 ** -23, 2.0 ** -19, 2.0 ** -22, 2.0 ** -17, 0.0,
             2.0 ** -11)
PREC_FP32 = (2.0 ** -21, 2.0 ** -23, 2.0 ** -22, 2.0 ** -22, 2.0 ** -24, 2.0 ** -22, 0.0, 2.0 ** -21, 0.0, 0.0)


def error_bounds(net: OracleNet, pts, prec, t: float = 0.0, grad=True):
    """First-order rounding-error bounds of a kernel path with precision
    model prec at each point: (B_out [n, D], B_grad [n, 3] or None)."""
    P = _d(pts).reshape(-1, 3)
    pr = _d(prec)
    Bo = np.zeros((len(P), net.dims["D"]))
    Bg = np.zeros((len(P), 3)) if grad else None
    lib().orc_error_bounds(C.byref(net.s), _p(P), len(P), _f32(t), _p(pr), _p(Bo), _p(Bg) if grad else None)
    return Bo, Bg


def fp16_grad_bound(net: OracleNet, pts, t: float = 0.0):
    """Per-component bound on the FP16 tensor-core adjoint gradient's error."""
    return error_bounds(net, pts, PREC_FP16, t)[1]


def render_shade_bound(net: OracleNet, cams, tf: OracleTF, W, H, step, et, shading, prec, fd_h=0.0, times=None,
                       pixels=None):
    """(rgba, bound): the oracle render and, per pixel, the bound on the
    shaded image's error that the gradient error of a kernel path with
    precision model prec causes (to be added to the unshaded image bound)."""
    T = 1 if times is None else len(times)
    tarr = None if times is None else _d32(times)
    pp, npix, keep = _pix(pixels)
    total = npix if pixels is not None else T * len(cams) * H * W
    out = np.zeros((total, 4))
    bound = np.zeros(total)
    pr = _d(prec)
    lib().orc_render_shade_bound(C.byref(net.s), _cams(cams), len(cams), _p(tarr) if tarr is not None else None, T,
                                 C.byref(tf.s), W, H, _f32(step), _f32(et), shading, _f32(fd_h), pp, npix, _p(pr),
                                 _p(out), _p(bound))
    if pixels is None:
        out = out.reshape(T, len(cams), H, W, 4)
        bound = bound.reshape(T, len(cams), H, W)
    return out, bound


def dvr_dense_shade_bound(vol, cams, tf: OracleTF, W, H, step, et, vol_abs, pixels=None):
    """(rgba, bound) of FD-shaded dense DVR whose volume samples are off by
    at most vol_abs."""
    v = _d(vol)
    nz, ny, nx = v.shape
    pp, npix, keep = _pix(pixels)
    total = npix if pixels is not None else len(cams) * H * W
    out = np.zeros((total, 4))
    bound = np.zeros(total)
    pr = _d((0, 0, 0, 0, 0, 0, 0, 0, vol_abs, 0))
    lib().orc_dvr_dense_shade_bound(_p(v), nx, ny, nz, _cams(cams), len(cams), C.byref(tf.s), W, H, _f32(step),
                                    _f32(et), pp,
                                    npix, _p(pr), _p(out), _p(bound))
    if pixels is None:
        out = out.reshape(len(cams), H, W, 4)
        bound = bound.reshape(len(cams), H, W)
    return out, bound
