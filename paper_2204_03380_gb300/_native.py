"""ctypes binding of librbc (include/rbc.h): argument marshalling only.

Every call checks tensor device/dtype/shape, passes raw pointers, the current
CUDA stream and host index arrays to the C ABI, and raises ``RBCError`` with
the library's message on a non-zero status.  There is no CPU fallback: if the
shared library has not been built, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librbc.so")

RBC_OK, RBC_EINVAL, RBC_ECFL, RBC_ENOMEM, RBC_ECUDA, RBC_ETIMEOUT, RBC_ENOTSUP = range(7)
RBC_REINJECT_SOURCE = 1
RBC_ZERO_FIRST = 2
_NAMES = {1: "EINVAL", 2: "ECFL", 3: "ENOMEM", 4: "ECUDA", 5: "ETIMEOUT", 6: "ENOTSUP"}


class RBCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"RBC_{_NAMES.get(code, code)}: {msg}")
        self.code = code


class rbc_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("nb", C.c_int), ("free_surface", C.c_int), ("h", C.c_double),
                ("dt", C.c_double), ("nt", C.c_int)]

    @property
    def top(self):
        """Rows above the interior: the random pad, or 4 zero-pressure rows with a free surface."""
        return 4 if self.free_surface else self.nb

    @property
    def padded(self):
        n = 2 * self.nb
        if self.ndim == 2:
            return (self.nz + self.nb + self.top, self.nx + n)
        return (self.nz + self.nb + self.top, self.ny + n, self.nx + n)

    @property
    def interior(self):
        return (self.nz, self.nx) if self.ndim == 2 else (self.nz, self.ny, self.nx)


class rbc_shot(C.Structure):
    _fields_ = [("src", C.c_int * 3), ("nrec", C.c_int), ("rec_host", C.c_void_p), ("seis_dev", C.c_void_p),
                ("off_x", C.c_int)]


def make_grid(ndim, nx, ny, nz, nb, h, dt, nt, free_surface=0) -> rbc_grid:
    return rbc_grid(int(ndim), int(nx), int(ny if ndim == 3 else 1), int(nz), int(nb),
                    int(free_surface), float(h), float(dt), int(nt))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librbc is not built ({LIB_PATH} missing): run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    P, I, F = C.c_void_p, C.c_int, C.c_float
    G = C.POINTER(rbc_grid)
    lib.rbc_build_velocity.argtypes = [G, P, F, F, F, C.c_uint64, I, P, P, P]
    lib.rbc_create.argtypes = [G, P, C.POINTER(C.c_void_p)]
    lib.rbc_destroy.argtypes = [P]
    lib.rbc_set_coef.argtypes = [P, P, I, P]
    lib.rbc_set_coef.restype = I
    lib.rbc_model.argtypes = [P, P, P, I, P, P, P]
    lib.rbc_rtm_shot.argtypes = [P, P, P, I, P, P, I, P, P, P]
    lib.rbc_image_stack.argtypes = [G, P, P, F, I, I, G, P, P]
    lib.rbc_nyquist_stride.argtypes = [C.c_double, C.c_double, C.c_double]
    lib.rbc_nyquist_stride.restype = I
    lib.rbc_storage_bytes.argtypes = [G, I]
    lib.rbc_storage_bytes.restype = C.c_longlong
    lib.rbc_rtm_storage.argtypes = [P, P, P, I, P, P, I, P, C.c_longlong, I, P, P, P]
    lib.rbc_set_snapshots.argtypes = [P, I, P, P, P, P]
    lib.rbc_get_panels.argtypes = [P, P, P, P]
    lib.rbc_phase_timing.argtypes = [P, I, P]
    lib.rbc_inject_fault.argtypes = [P, I]
    lib.rbc_inject_fault.restype = I
    lib.rbc_fwi_forward.argtypes = [P, P, P, I, P, P, P, P, P, P]
    lib.rbc_fwi_backward.argtypes = [P, P, P, I, P, P, P, P, P]
    lib.rbc_fwi_forward.restype = I
    lib.rbc_fwi_backward.restype = I
    lib.rbc_batch_create.argtypes = [G, I, P, P, C.POINTER(C.c_void_p)]
    lib.rbc_batch_destroy.argtypes = [P]
    lib.rbc_batch_rtm.argtypes = [P, P, P, I, F, P, I, P]
    lib.rbc_batch_info.argtypes = [P, P]
    lib.rbc_batch_timing.argtypes = [P, I, P]
    for name in ("rbc_batch_create", "rbc_batch_destroy", "rbc_batch_rtm", "rbc_batch_info", "rbc_batch_timing"):
        getattr(lib, name).restype = I
    lib.rbc_cnn_param_count.restype = C.c_longlong
    lib.rbc_cnn_param_count.argtypes = []
    lib.rbc_cnn_workspace_bytes.restype = C.c_longlong
    lib.rbc_cnn_workspace_bytes.argtypes = [I, I, I]
    lib.rbc_cnn_forward.argtypes = [P, I, I, I, P, P, P, P]
    lib.rbc_cnn_infer.argtypes = [P, I, I, I, P, P, P, P]
    lib.rbc_cnn_backward.argtypes = [P, I, I, I, P, P, P, P]
    lib.rbc_cnn_mse.argtypes = [P, P, C.c_longlong, P, P, P]
    lib.rbc_cnn_adam.argtypes = [P, P, P, P, F, F, F, F, I, P]
    for name in ("rbc_cnn_forward", "rbc_cnn_infer", "rbc_cnn_backward", "rbc_cnn_mse", "rbc_cnn_adam"):
        getattr(lib, name).restype = I
    lib.rbc_model_static.argtypes = [G, P, P, P, I, P, P, P]
    lib.rbc_model_static.restype = I
    lib.rbc_last_error.restype = C.c_char_p
    lib.rbc_launch_count.argtypes = [I]
    lib.rbc_launch_count.restype = C.c_longlong
    for name in ("rbc_build_velocity", "rbc_create", "rbc_destroy", "rbc_model", "rbc_rtm_shot",
                 "rbc_image_stack", "rbc_set_snapshots", "rbc_get_panels", "rbc_phase_timing"):
        getattr(lib, name).restype = I
    return lib


_lib = _load()
EXPORTED = ("rbc_build_velocity", "rbc_create", "rbc_destroy", "rbc_model", "rbc_rtm_shot",
            "rbc_image_stack", "rbc_set_snapshots", "rbc_get_panels", "rbc_phase_timing",
            "rbc_model_static", "rbc_fwi_forward", "rbc_fwi_backward", "rbc_batch_create",
            "rbc_batch_destroy", "rbc_batch_rtm", "rbc_batch_info", "rbc_batch_timing",
            "rbc_cnn_param_count", "rbc_cnn_workspace_bytes", "rbc_cnn_forward", "rbc_cnn_infer", "rbc_cnn_backward",
            "rbc_cnn_mse", "rbc_cnn_adam", "rbc_inject_fault", "rbc_last_error",
            "rbc_launch_count", "rbc_nyquist_stride", "rbc_storage_bytes", "rbc_rtm_storage",
            "rbc_set_coef")


def _check(code):
    if code != RBC_OK:
        raise RBCError(code, _lib.rbc_last_error().decode())


def _dev(t, shape=None, name="tensor"):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _nodes(a, n=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1, 3))
    if n is not None and arr.shape[0] != n:
        raise ValueError("bad node list")
    return arr


def rbc_build_velocity(grid, v_int, v_lo, v_hi, v_max, seed, mode, v_pad, a, stream=None):
    _check(_lib.rbc_build_velocity(C.byref(grid), _dev(v_int, grid.interior, "v_int"), float(v_lo),
                                   float(v_hi), float(v_max), C.c_uint64(int(seed)), int(mode),
                                   _dev(v_pad, grid.padded, "v_pad"), _dev(a, grid.padded, "a"),
                                   _stream(stream)))


def rbc_create(grid, a):
    """Returns an opaque context handle (int); free it with rbc_destroy."""
    out = C.c_void_p()
    torch.cuda.synchronize()
    _check(_lib.rbc_create(C.byref(grid), _dev(a, grid.padded, "a"), C.byref(out)))
    return out.value


def rbc_destroy(ctx):
    _check(_lib.rbc_destroy(C.c_void_p(ctx)))


def rbc_set_coef(ctx, grid, a, check=True, stream=None):
    """Replace the context's padded coefficient a (grid.padded fp32 CUDA)."""
    _check(_lib.rbc_set_coef(C.c_void_p(ctx), _dev(a, grid.padded, "a"), int(bool(check)), _stream(stream)))


def rbc_model(ctx, src, wavelet, rec, seis, stream=None):
    s = _nodes(src, 1)
    r = _nodes(rec)
    _check(_lib.rbc_model(C.c_void_p(ctx), s.ctypes.data_as(C.c_void_p), _dev(wavelet, None, "wavelet"),
                          r.shape[0], r.ctypes.data_as(C.c_void_p) if r.size else None,
                          _dev(seis, None, "seis") if r.shape[0] else None, _stream(stream)))


def rbc_rtm_shot(ctx, src, wavelet, rec, seis, flags, num, den, stream=None):
    s = _nodes(src, 1)
    r = _nodes(rec)
    _check(_lib.rbc_rtm_shot(C.c_void_p(ctx), s.ctypes.data_as(C.c_void_p), _dev(wavelet, None, "wavelet"),
                             r.shape[0], r.ctypes.data_as(C.c_void_p) if r.size else None,
                             _dev(seis, None, "seis") if r.shape[0] else None, int(flags),
                             _dev(num, None, "num"), _dev(den, None, "den"), _stream(stream)))


def rbc_nyquist_stride(dt, f_max, f_min=0.0) -> int:
    k = int(_lib.rbc_nyquist_stride(float(dt), float(f_max), float(f_min)))
    if k < 1:
        raise RBCError(RBC_EINVAL, _lib.rbc_last_error().decode())
    return k


def rbc_storage_bytes(grid, stride) -> int:
    n = int(_lib.rbc_storage_bytes(C.byref(grid), int(stride)))
    if n < 0:
        raise RBCError(RBC_EINVAL, _lib.rbc_last_error().decode())
    return n


def rbc_rtm_storage(ctx, src, wavelet, rec, seis, stride, store, flags, num, den, stream=None):
    """store: contiguous fp32 CUDA tensor of at least rbc_storage_bytes(grid, stride) bytes."""
    s = _nodes(src, 1)
    r = _nodes(rec)
    if not (isinstance(store, torch.Tensor) and store.is_cuda and store.dtype == torch.float32
            and store.is_contiguous()):
        raise TypeError("store must be a contiguous float32 CUDA tensor")
    _check(_lib.rbc_rtm_storage(C.c_void_p(ctx), s.ctypes.data_as(C.c_void_p), _dev(wavelet, None, "wavelet"),
                                r.shape[0], r.ctypes.data_as(C.c_void_p) if r.size else None,
                                _dev(seis, None, "seis") if r.shape[0] else None, int(stride),
                                C.c_void_p(store.data_ptr()), store.numel() * 4, int(flags),
                                _dev(num, None, "num"), _dev(den, None, "den"), _stream(stream)))


def rbc_image_stack(shot_grid, num, den, eps_rel, off_x, off_y, survey_grid, image, stream=None):
    _check(_lib.rbc_image_stack(C.byref(shot_grid), _dev(num, shot_grid.interior, "num"),
                                _dev(den, shot_grid.interior, "den"), float(eps_rel), int(off_x), int(off_y),
                                C.byref(survey_grid), _dev(image, survey_grid.interior, "image"),
                                _stream(stream)))


def rbc_set_snapshots(ctx, levels, pf=None, pr=None, pb=None):
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32).ravel())
    _check(_lib.rbc_set_snapshots(C.c_void_p(ctx), lv.size, lv.ctypes.data_as(C.c_void_p) if lv.size else None,
                                  _dev(pf, None, "pf"), _dev(pr, None, "pr"), _dev(pb, None, "pb")))


def rbc_get_panels(ctx, prev=None, last=None, stream=None):
    _check(_lib.rbc_get_panels(C.c_void_p(ctx), _dev(prev, None, "prev"), _dev(last, None, "last"),
                               _stream(stream)))


def rbc_phase_timing(ctx, enable):
    """enable=True starts phase timing; enable=False stops and returns
    dict(fwd_ms, rev_ms, fwd_launches, rev_launches, shots)."""
    out = (C.c_double * 5)()
    _check(_lib.rbc_phase_timing(C.c_void_p(ctx), 1 if enable else 0, out))
    if enable:
        return None
    return dict(fwd_ms=out[0], rev_ms=out[1], fwd_launches=int(out[2]), rev_launches=int(out[3]),
                shots=int(out[4]))


def rbc_model_static(grid, a, src, wavelet, rec, seis, stream=None):
    """Modeling without a context and without any device allocation: the
    scratch is the library's fixed 16 MiB per-device workspace (for callers
    that cannot call cudaMalloc).  Calls sharing a device must not overlap."""
    s = _nodes(src, 1)
    r = _nodes(rec)
    _check(_lib.rbc_model_static(C.byref(grid), _dev(a, grid.padded, "a"), s.ctypes.data_as(C.c_void_p),
                                 _dev(wavelet, None, "wavelet"), r.shape[0],
                                 r.ctypes.data_as(C.c_void_p) if r.size else None,
                                 _dev(seis, None, "seis") if r.shape[0] else None, _stream(stream)))


def rbc_fwi_forward(ctx, src, wavelet, rec, dobs, resid, misfit, panels=None, stream=None):
    """misfit (float64 CUDA tensor of one element) += 1/2 ||record - dobs||^2;
    resid = record - dobs; panels (2, *padded) receives p^{nt-1}, p^{nt}."""
    s = _nodes(src, 1)
    r = _nodes(rec)
    if not (misfit.is_cuda and misfit.dtype == torch.float64 and misfit.numel() == 1):
        raise TypeError("misfit must be a one-element float64 CUDA tensor")
    _check(_lib.rbc_fwi_forward(C.c_void_p(ctx), s.ctypes.data_as(C.c_void_p), _dev(wavelet, None, "wavelet"),
                                r.shape[0], r.ctypes.data_as(C.c_void_p), _dev(dobs, None, "dobs"),
                                _dev(resid, None, "resid"), C.c_void_p(misfit.data_ptr()),
                                _dev(panels, None, "panels"), _stream(stream)))


def rbc_fwi_backward(ctx, src, wavelet, rec, resid, panels, grad, stream=None):
    """grad (interior) += dJ/dv by the adjoint, from the residual and the two panels."""
    s = _nodes(src, 1)
    r = _nodes(rec)
    _check(_lib.rbc_fwi_backward(C.c_void_p(ctx), s.ctypes.data_as(C.c_void_p), _dev(wavelet, None, "wavelet"),
                                 r.shape[0], r.ctypes.data_as(C.c_void_p), _dev(resid, None, "resid"),
                                 _dev(panels, None, "panels"), _dev(grad, None, "grad"), _stream(stream)))


def rbc_batch_create(grid, nx_list, a_list):
    """Batch of 2-D shots sharing grid's nz/nb/h/dt/nt with widths nx_list and
    padded coefficients a_list (one CUDA tensor per shot).  Returns a handle."""
    n = len(nx_list)
    nx = (C.c_int * n)(*[int(x) for x in nx_list])
    ptrs = (C.c_void_p * n)()
    for k, (x, a) in enumerate(zip(nx_list, a_list)):
        ptrs[k] = _dev(a, (grid.nz + 2 * grid.nb, int(x) + 2 * grid.nb), "a")
    out = C.c_void_p()
    torch.cuda.synchronize()
    _check(_lib.rbc_batch_create(C.byref(grid), n, nx, ptrs, C.byref(out)))
    return out.value


def rbc_batch_destroy(batch):
    _check(_lib.rbc_batch_destroy(C.c_void_p(batch)))


def rbc_batch_rtm(batch, shots, wavelet, flags, eps_rel, image, stream=None):
    """shots: list of dict(src=(x, 0, z), rec=(nrec, 3) int array, seis=(nrec, nt+1)
    CUDA tensor, off_x=int).  image: survey interior (nz, survey_nx), += stacked."""
    n = len(shots)
    arr = (rbc_shot * n)()
    keep = []
    for k, sh in enumerate(shots):
        r = _nodes(sh["rec"])
        keep.append(r)
        arr[k].src[:] = [int(x) for x in np.asarray(sh["src"]).ravel()[:3]]
        arr[k].nrec = r.shape[0]
        arr[k].rec_host = r.ctypes.data if r.size else None
        arr[k].seis_dev = _dev(sh["seis"], None, "seis").value if r.shape[0] else None
        arr[k].off_x = int(sh["off_x"])
    _check(_lib.rbc_batch_rtm(C.c_void_p(batch), arr, _dev(wavelet, None, "wavelet"), int(flags),
                              float(eps_rel), _dev(image, None, "image"), int(image.shape[-1]),
                              _stream(stream)))


def rbc_batch_timing(batch, enable):
    """Phase timing of rbc_batch_rtm calls (see rbc_phase_timing)."""
    out = (C.c_double * 5)()
    _check(_lib.rbc_batch_timing(C.c_void_p(batch), 1 if enable else 0, out))
    if enable:
        return None
    return dict(fwd_ms=out[0], rev_ms=out[1], fwd_launches=int(out[2]), rev_launches=int(out[3]),
                calls=int(out[4]))


def rbc_batch_info(batch):
    out = (C.c_int * 15)()
    _check(_lib.rbc_batch_info(C.c_void_p(batch), out))
    return dict(rows_fwd=out[0], rows_rev=out[1], items_fwd=out[2], items_rev=out[3], grid_fwd=out[4],
                grid_rev=out[5], tune_us={"fwd_stream": out[6], "fwd_1": out[7], "fwd_2": out[8], "fwd_4": out[9],
                                          "rev_1": out[10], "rev_2": out[11], "rev_stream": out[12],
                                          "rev_tile": out[13]},
                groups=out[14])


def rbc_cnn_param_count() -> int:
    return int(_lib.rbc_cnn_param_count())


def rbc_cnn_workspace_bytes(nimg, H, W) -> int:
    return int(_lib.rbc_cnn_workspace_bytes(int(nimg), int(H), int(W)))


def _u8(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def rbc_cnn_forward(params, x, y, ws, stream=None):
    """x, y: (nimg, H, W) fp32; ws: uint8 workspace of rbc_cnn_workspace_bytes."""
    n, H, W = x.shape
    _check(_lib.rbc_cnn_forward(_dev(params, None, "params"), n, H, W, _dev(x, None, "x"), _dev(y, None, "y"),
                                _u8(ws, "ws"), _stream(stream)))


def rbc_cnn_infer(params, x, y, ws, stream=None):
    """Inference forward (keeps nothing for a backward pass); arguments as rbc_cnn_forward."""
    n, H, W = x.shape
    _check(_lib.rbc_cnn_infer(_dev(params, None, "params"), n, H, W, _dev(x, None, "x"), _dev(y, None, "y"),
                              _u8(ws, "ws"), _stream(stream)))


def rbc_cnn_backward(params, dy, grad, ws, stream=None):
    n, H, W = dy.shape
    _check(_lib.rbc_cnn_backward(_dev(params, None, "params"), n, H, W, _dev(dy, None, "dy"),
                                 _dev(grad, None, "grad"), _u8(ws, "ws"), _stream(stream)))


def rbc_cnn_mse(y, t, dy, loss, stream=None):
    _check(_lib.rbc_cnn_mse(_dev(y, None, "y"), _dev(t, None, "t"), y.numel(),
                            _dev(dy, None, "dy") if dy is not None else None, _u8(loss, "loss"), _stream(stream)))


def rbc_cnn_adam(params, grad, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _check(_lib.rbc_cnn_adam(_dev(params, None, "params"), _dev(grad, None, "grad"), _dev(m, None, "m"),
                             _dev(v, None, "v"), float(lr), float(b1), float(b2), float(eps), int(step),
                             _stream(stream)))


def rbc_inject_fault(ctx, mode=1):
    """Test hook: make the next call's first 3-D forward launch run a bounded
    wait out (see include/rbc.h); the call after it reports RBC_ETIMEOUT.
    ctx = None arms the next 3-D rbc_model_static call instead."""
    _check(_lib.rbc_inject_fault(C.c_void_p(ctx), int(mode)))


def rbc_last_error() -> str:
    return _lib.rbc_last_error().decode()


def rbc_launch_count(reset: bool = False) -> int:
    return int(_lib.rbc_launch_count(1 if reset else 0))
