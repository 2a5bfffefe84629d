"""Thin ctypes binding of the C ABI in ``include/srn.h``.

Functions carry the C names and only marshal arguments (torch tensors ->
device pointers, Python lists -> C structs, streams -> ``cudaStream_t``).
Every computation runs in the CUDA library ``libsrn.so``; there is no CPU
fallback: importing the binding on a machine without the built library
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsrn.so")

SRN_OK, SRN_ERR_INVALID_ARG, SRN_ERR_UNSUPPORTED, SRN_ERR_CUDA, SRN_ERR_NONFINITE, SRN_ERR_TIMEOUT, \
    SRN_ERR_INTERNAL = range(7)
SRN_ACT_SINE, SRN_ACT_SNAKEALT = 0, 1
SRN_PREC_FP32, SRN_PREC_FP16, SRN_PREC_BF16 = 0, 1, 2
SRN_SHADE_NONE, SRN_SHADE_ADJOINT, SRN_SHADE_FD, SRN_SHADE_HEAD = 0, 1, 2, 3
SRN_MAX_KEYFRAMES, SRN_MAX_TF_POINTS, SRN_MAX_VIEWS, SRN_MAX_TIMES = 32, 32, 64, 64

EXPORTED = ["srn_version", "srn_last_error", "srn_create", "srn_destroy", "srn_set_params", "srn_sync_half",
            "srn_render", "srn_dvr_dense", "srn_eval", "srn_density_grad", "srn_backward", "srn_fit_step",
            "srn_sync_status", "srn_image_mse", "srn_backward_static", "srn_density_mse", "srn_resample",
            "srn_lowpass_resample", "srn_save", "srn_load", "srn_error_grid", "srn_fit_set_sampling",
            "srn_fit_points", "srn_fit_steps", "srn_image_ssim", "srn_input_backward"]


class SrnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"srn status {status}: {msg}")
        self.status = status


class srn_config(C.Structure):
    _fields_ = [("grid_res", C.c_int), ("feat", C.c_int), ("n_fourier", C.c_int), ("layers", C.c_int),
                ("width", C.c_int), ("out_dim", C.c_int), ("activation", C.c_int), ("precision", C.c_int),
                ("n_keyframes", C.c_int), ("key_times", C.c_float * SRN_MAX_KEYFRAMES),
                ("max_fit_points", C.c_int), ("time_input", C.c_int), ("grid_u8", C.c_int)]


class srn_params(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("fourier", C.c_void_p), ("weights", C.c_void_p), ("biases", C.c_void_p),
                ("grid_h", C.c_void_p), ("weights_h", C.c_void_p), ("adam_m", C.c_void_p),
                ("adam_v", C.c_void_p), ("grid_q", C.c_void_p), ("grid_qp", C.c_void_p)]


class srn_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("fovy", C.c_float)]


class srn_tf(C.Structure):
    _fields_ = [("n", C.c_int), ("pos", C.POINTER(C.c_float)), ("rgba", C.POINTER(C.c_float)),
                ("opacity_scale", C.c_float)]


class srn_render_desc(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("step", C.c_float), ("et_threshold", C.c_float),
                ("shading", C.c_int), ("fd_h", C.c_float)]


_lib = None


def lib():
    """Load libsrn.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, i, f = C.c_void_p, C.c_int, C.c_float
        L.srn_version.restype = C.c_char_p
        L.srn_last_error.restype = C.c_char_p
        L.srn_create.argtypes = [C.POINTER(srn_config), C.POINTER(srn_params), C.POINTER(vp)]
        L.srn_destroy.argtypes = [vp]
        L.srn_set_params.argtypes = [vp, C.POINTER(srn_params)]
        L.srn_sync_half.argtypes = [vp, vp]
        L.srn_render.argtypes = [vp, C.POINTER(srn_camera), i, C.POINTER(C.c_float), i, C.POINTER(srn_tf),
                                 C.POINTER(srn_render_desc), vp, vp, vp]
        L.srn_dvr_dense.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(srn_camera), i, C.POINTER(srn_tf),
                                    C.POINTER(srn_render_desc), vp, vp, vp]
        L.srn_eval.argtypes = [vp, vp, i, f, vp, vp]
        L.srn_density_grad.argtypes = [vp, vp, i, f, vp, vp, vp]
        L.srn_input_backward.argtypes = [vp, vp, i, f, vp, vp, vp]
        L.srn_backward.argtypes = [vp, vp, i, f, vp, vp, vp, vp, vp]
        L.srn_fit_step.argtypes = [vp, vp, C.POINTER(C.c_int), i, C.c_uint64, i, f, f, f, f, f, vp, vp]
        L.srn_sync_status.argtypes = [vp, vp]
        L.srn_image_mse.argtypes = [vp, vp, C.c_longlong, vp, vp]
        L.srn_backward_static.argtypes = [C.POINTER(srn_config), C.POINTER(srn_params), vp, i, f, vp, vp, vp, vp,
                                          vp]
        L.srn_density_mse.argtypes = [vp, vp, C.c_longlong, vp, vp]
        L.srn_resample.argtypes = [vp, C.POINTER(C.c_int), vp, C.POINTER(C.c_int), vp]
        L.srn_lowpass_resample.argtypes = [vp, C.POINTER(C.c_int), i, vp, vp, vp]
        L.srn_save.argtypes = [vp, C.c_char_p, i]
        L.srn_load.argtypes = [vp, C.c_char_p, C.POINTER(C.c_int)]
        L.srn_error_grid.argtypes = [vp, vp, C.POINTER(C.c_int), i, i, C.c_uint64, f, vp, vp]
        L.srn_fit_set_sampling.argtypes = [vp, vp, i, vp]
        L.srn_fit_points.argtypes = [vp, i, C.c_uint64, i, vp, vp]
        L.srn_fit_steps.argtypes = [vp, vp, C.POINTER(C.c_int), i, C.c_uint64, i, i, f, f, f, f, f, vp, vp]
        L.srn_image_ssim.argtypes = [vp, vp, i, i, vp, vp]
        for name in EXPORTED[2:]:
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(st):
    if st != SRN_OK:
        raise SrnError(st, lib().srn_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _cams(cams):
    arr = (srn_camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k].eye[:] = [float(x) for x in c["eye"]]
        arr[k].target[:] = [float(x) for x in c["target"]]
        arr[k].up[:] = [float(x) for x in c["up"]]
        arr[k].fovy = float(c["fovy"])
    return arr


def make_tf(tf):
    pos = np.ascontiguousarray(np.asarray(tf["pos"], np.float32))
    rgba = np.ascontiguousarray(np.asarray(tf["rgba"], np.float32).reshape(-1))
    s = srn_tf(len(pos), pos.ctypes.data_as(C.POINTER(C.c_float)), rgba.ctypes.data_as(C.POINTER(C.c_float)),
               float(tf["opacity_scale"]))
    s._keep = (pos, rgba)
    return s


def render_desc(width, height, step, et_threshold=0.99, shading=SRN_SHADE_NONE, fd_h=0.0):
    return srn_render_desc(int(width), int(height), float(step), float(et_threshold), int(shading), float(fd_h))


def srn_version() -> str:
    return lib().srn_version().decode()


def srn_last_error() -> str:
    return lib().srn_last_error().decode()


def srn_create(cfg: srn_config, params: srn_params):
    h = C.c_void_p()
    _check(lib().srn_create(C.byref(cfg), C.byref(params), C.byref(h)))
    return h


def srn_destroy(ctx):
    _check(lib().srn_destroy(ctx))


def srn_set_params(ctx, params: srn_params):
    _check(lib().srn_set_params(ctx, C.byref(params)))


def srn_sync_half(ctx, stream=None):
    _check(lib().srn_sync_half(ctx, _stream(stream)))


def srn_render(ctx, cams, tf, desc, rgba, times=None, samples=None, stream=None):
    """rgba: float32 CUDA tensor [T, V, H, W, 4]; samples: uint64/int64 [1] or None."""
    tarr = None if times is None else (C.c_float * len(times))(*[float(t) for t in times])
    _check(lib().srn_render(ctx, _cams(cams), len(cams), tarr, 1 if times is None else len(times),
                            C.byref(make_tf(tf) if isinstance(tf, dict) else tf), C.byref(desc), _ptr(rgba),
                            _ptr(samples), _stream(stream)))


def srn_dvr_dense(volume, cams, tf, desc, rgba, samples=None, stream=None):
    """volume: float32 CUDA tensor [nz, ny, nx]."""
    nz, ny, nx = volume.shape
    dims = (C.c_int * 3)(nx, ny, nz)
    _check(lib().srn_dvr_dense(_ptr(volume), dims, _cams(cams), len(cams),
                               C.byref(make_tf(tf) if isinstance(tf, dict) else tf), C.byref(desc), _ptr(rgba),
                               _ptr(samples), _stream(stream)))


def srn_eval(ctx, pts, out, time=0.0, stream=None):
    _check(lib().srn_eval(ctx, _ptr(pts), pts.shape[0], float(time), _ptr(out), _stream(stream)))


def srn_density_grad(ctx, pts, rho, grad=None, time=0.0, stream=None):
    _check(lib().srn_density_grad(ctx, _ptr(pts), pts.shape[0], float(time), _ptr(rho), _ptr(grad),
                                  _stream(stream)))


def srn_input_backward(ctx, pts, dout, dpts, time=0.0, stream=None):
    """dpts [n, 3] = sum_d dout[:, d] * d out_d / d p (overwritten)."""
    _check(lib().srn_input_backward(ctx, _ptr(pts), pts.shape[0], float(time), _ptr(dout), _ptr(dpts),
                                    _stream(stream)))


def srn_backward(ctx, pts, dout, dgrid, dweights, dbiases, time=0.0, stream=None):
    _check(lib().srn_backward(ctx, _ptr(pts), pts.shape[0], float(time), _ptr(dout), _ptr(dgrid), _ptr(dweights),
                              _ptr(dbiases), _stream(stream)))


def srn_backward_static(cfg, params, pts, dout, dgrid, dweights, dbiases, time=0.0, stream=None):
    """srn_backward without a context and without any device allocation (a
    fixed device array inside the library); for callers that may not
    allocate, e.g. hosts whose device memory belongs to another allocator."""
    _check(lib().srn_backward_static(C.byref(cfg), C.byref(params), _ptr(pts), pts.shape[0], float(time),
                                     _ptr(dout), _ptr(dgrid), _ptr(dweights), _ptr(dbiases), _stream(stream)))


def srn_error_grid(ctx, volume, res, samples_per_voxel, seed, err, time=0.0, stream=None):
    """Section 6.2 error grid: err float32 CUDA tensor of res^3 entries."""
    nz, ny, nx = volume.shape
    dims = (C.c_int * 3)(nx, ny, nz)
    _check(lib().srn_error_grid(ctx, _ptr(volume), dims, int(res), int(samples_per_voxel), int(seed), float(time),
                                _ptr(err), _stream(stream)))


def srn_fit_set_sampling(ctx, err, res=0, stream=None):
    """Draw later fit points in proportion to err (res^3 float32 CUDA
    tensor); err=None returns to uniform sampling."""
    _check(lib().srn_fit_set_sampling(ctx, None if err is None else _ptr(err), int(res), _stream(stream)))


def srn_fit_points(ctx, n_points, seed, step, pts, stream=None):
    _check(lib().srn_fit_points(ctx, int(n_points), int(seed), int(step), _ptr(pts), _stream(stream)))


def srn_fit_step(ctx, volume, n_points, seed, step, loss, lr_grid=1e-2, lr_net=5e-3, time=0.0, grad_weight=0.0,
                 grad_scale=1.0, stream=None):
    nz, ny, nx = volume.shape
    dims = (C.c_int * 3)(nx, ny, nz)
    _check(lib().srn_fit_step(ctx, _ptr(volume), dims, int(n_points), int(seed), int(step), float(time),
                              float(lr_grid), float(lr_net), float(grad_weight), float(grad_scale), _ptr(loss),
                              _stream(stream)))


def srn_fit_steps(ctx, volume, n_points, seed, first_step, n_steps, loss, lr_grid=1e-2, lr_net=5e-3, time=0.0,
                  grad_weight=0.0, grad_scale=1.0, stream=None):
    nz, ny, nx = volume.shape
    dims = (C.c_int * 3)(nx, ny, nz)
    _check(lib().srn_fit_steps(ctx, _ptr(volume), dims, int(n_points), int(seed), int(first_step), int(n_steps),
                               float(time), float(lr_grid), float(lr_net), float(grad_weight), float(grad_scale),
                               _ptr(loss), _stream(stream)))


def srn_sync_status(ctx, stream=None):
    st = lib().srn_sync_status(ctx, _stream(stream))
    return st, (srn_last_error() if st else "")


def srn_image_mse(a, b, out, stream=None):
    """out: float64 CUDA tensor [1]."""
    _check(lib().srn_image_mse(_ptr(a), _ptr(b), a.numel() // 4, _ptr(out), _stream(stream)))


def srn_save(ctx, path, step):
    _check(lib().srn_save(ctx, str(path).encode(), int(step)))


def srn_load(ctx, path):
    """Returns the step stored in the checkpoint."""
    st = C.c_int()
    _check(lib().srn_load(ctx, str(path).encode(), C.byref(st)))
    return st.value


def srn_image_ssim(a, b, out, stream=None):
    """a, b: [H, W, 4] float32 CUDA images; out: float64 CUDA tensor [1]."""
    H, W = a.shape[-3], a.shape[-2]
    _check(lib().srn_image_ssim(_ptr(a), _ptr(b), int(W), int(H), _ptr(out), _stream(stream)))


def srn_density_mse(a, b, out, stream=None):
    """out: float64 CUDA tensor [1]."""
    _check(lib().srn_density_mse(_ptr(a), _ptr(b), a.numel(), _ptr(out), _stream(stream)))


def _dims(t):
    nz, ny, nx = t.shape
    return (C.c_int * 3)(nx, ny, nz)


def srn_resample(src, dst, stream=None):
    """src, dst: float32 CUDA tensors [nz, ny, nx]."""
    _check(lib().srn_resample(_ptr(src), _dims(src), _ptr(dst), _dims(dst), _stream(stream)))


def srn_lowpass_resample(volume, M, tmp, out, stream=None):
    """tmp: float32 CUDA tensor with 2 * volume.numel() values; out: [M, M, M]."""
    _check(lib().srn_lowpass_resample(_ptr(volume), _dims(volume), int(M), _ptr(tmp), _ptr(out), _stream(stream)))


# --------------------------------------------------------------------------
class Network:
    """Device-resident fV-SRN parameters (torch CUDA tensors) plus a context.

    Packs a parameter dict (``grid`` [nkey, R, R, R, F], ``fourier`` [m, 3],
    ``weights`` list of [d_out, d_in], ``biases`` list, ``act``,
    ``key_times``) into the flat layouts of ``srn_params``.
    """

    def __init__(self, params: dict, precision=SRN_PREC_FP32, max_fit_points=0, device="cuda", adam=False,
                 grid_u8=False):
        import torch
        g = np.asarray(params["grid"], np.float32)
        self.nkey, self.R = g.shape[0], g.shape[1]
        self.F = g.shape[4]
        Ws = [np.asarray(w, np.float32) for w in params["weights"]]
        bs = [np.asarray(b, np.float32) for b in params["biases"]]
        self.m = np.asarray(params["fourier"]).shape[0]
        self.layers, self.width, self.out_dim = len(Ws), Ws[0].shape[0], Ws[-1].shape[0]
        self.layer_shapes = [w.shape for w in Ws]
        dev = torch.device(device)
        self.grid = torch.tensor(g.reshape(-1), device=dev)
        self.fourier = torch.tensor(np.asarray(params["fourier"], np.float32).reshape(-1), device=dev)
        self.weights = torch.tensor(np.concatenate([w.reshape(-1) for w in Ws]), device=dev)
        self.biases = torch.tensor(np.concatenate(bs), device=dev)
        self.grid_h = torch.empty(self.grid.numel(), dtype=torch.float16, device=dev)
        self.weights_h = torch.empty(self.weights.numel(), dtype=torch.float16, device=dev)
        self.grid_q = torch.zeros(self.grid.numel(), dtype=torch.uint8, device=dev) if grid_u8 else None
        self.grid_qp = torch.zeros((self.F, 2), dtype=torch.float32, device=dev) if grid_u8 else None
        n_par = self.grid.numel() + self.weights.numel() + self.biases.numel()
        self.adam_m = torch.zeros(n_par, device=dev) if adam else None
        self.adam_v = torch.zeros(n_par, device=dev) if adam else None
        cfg = srn_config()
        cfg.grid_res, cfg.feat, cfg.n_fourier, cfg.layers = self.R, self.F, self.m, self.layers
        cfg.width, cfg.out_dim, cfg.activation, cfg.precision = self.width, self.out_dim, int(params["act"]), precision
        cfg.n_keyframes = self.nkey
        kt = list(np.asarray(params.get("key_times", np.arange(self.nkey)), np.float32))
        for k in range(self.nkey):
            cfg.key_times[k] = float(kt[k])
        cfg.max_fit_points = int(max_fit_points)
        cfg.time_input = int(params.get("time_input", 0))
        cfg.grid_u8 = 1 if grid_u8 else 0
        self.cfg = cfg
        self.ctx = srn_create(cfg, self._params())
        srn_sync_half(self.ctx)

    def _params(self):
        p = srn_params()
        p.grid, p.fourier = self.grid.data_ptr(), self.fourier.data_ptr()
        p.weights, p.biases = self.weights.data_ptr(), self.biases.data_ptr()
        p.grid_h, p.weights_h = self.grid_h.data_ptr(), self.weights_h.data_ptr()
        if self.adam_m is not None:
            p.adam_m, p.adam_v = self.adam_m.data_ptr(), self.adam_v.data_ptr()
        if self.grid_q is not None:
            p.grid_q, p.grid_qp = self.grid_q.data_ptr(), self.grid_qp.data_ptr()
        return p

    def unpack(self):
        """Current parameters as a numpy dict (FP32 masters)."""
        W = self.weights.cpu().numpy()
        b = self.biases.cpu().numpy()
        Ws, bs, o, ob = [], [], 0, 0
        for s in self.layer_shapes:
            Ws.append(W[o:o + s[0] * s[1]].reshape(s))
            bs.append(b[ob:ob + s[0]])
            o += s[0] * s[1]
            ob += s[0]
        return dict(grid=self.grid.cpu().numpy().reshape(self.nkey, self.R, self.R, self.R, self.F),
                    fourier=self.fourier.cpu().numpy().reshape(-1, 3), weights=Ws, biases=bs,
                    act=self.cfg.activation, key_times=np.array(self.cfg.key_times[:self.nkey], np.float32),
                    time_input=int(self.cfg.time_input))

    def unpack_half(self):
        """The FP16 copies widened to float32 (what the FP16 path computes with)."""
        d = self.unpack()
        gh = self.grid_h.float().cpu().numpy().reshape(d["grid"].shape)
        Wh = self.weights_h.float().cpu().numpy()
        Ws, o = [], 0
        for s in self.layer_shapes:
            Ws.append(Wh[o:o + s[0] * s[1]].reshape(s))
            o += s[0] * s[1]
        d["grid"], d["weights"] = gh, Ws
        return d

    def unpack_u8(self):
        """Parameters as the 8-bit FP16 path sees them: the dequantized grid
        lo + step * code (float64 -> float32 exact for these values is not
        needed: the oracle takes float64), FP16 weights."""
        d = self.unpack_half()
        q = self.grid_q.cpu().numpy().astype(np.float64).reshape(-1, self.F)
        qp = self.grid_qp.cpu().numpy().astype(np.float64)
        g = qp[None, :, 0] + qp[None, :, 1] * q
        d["grid"] = g.reshape(self.nkey, self.R, self.R, self.R, self.F)
        return d

    def close(self):
        if self.ctx is not None:
            srn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
