"""FP64 CPU oracle for RTM with random boundary conditions (arXiv:2204.03380).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import this package.  It shares
no code with the CUDA library (``paper_2204_03380_gb300``) and never imports it.

The arithmetic lives in ``rbc_oracle.c`` (plain C, fp64, OpenMP over the outer
axis); this module compiles it with gcc and marshals numpy arrays.  Each
wrapper names the passage of the paper it follows; the C file states the
recursion in full.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

REC_SIGN = 1.0  # sign of the back-propagated data (pinned by the flat-reflector test)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march flags: builds on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i, u64 = C.c_double, C.c_int, C.c_uint64
            P = C.c_void_p
            lib.orc_leapfrog.argtypes = [i, i, i, i, P, P, P, P]
            lib.orc_lap8_point.argtypes = [i, i, i, i, P, i, i, i]
            lib.orc_lap8_point.restype = d
            lib.orc_model.argtypes = [i, i, i, i, P, d, i, P, P, i, P, P, P, P, i, P, P]
            lib.orc_model.restype = i
            lib.orc_rtm_shot.argtypes = [i, i, i, i, P, d, i, P, P, i, P, P, i, d,
                                         i, i, i, i, i, P, P, i, P, P, P]
            lib.orc_rtm_shot.restype = i
            lib.orc_rtm_storage.argtypes = [i, i, i, i, P, d, i, P, P, i, P, P, d, i,
                                            i, i, i, i, i, P, P, P]
            lib.orc_rtm_storage.restype = i
            lib.orc_nyquist_stride.argtypes = [d, d, d]
            lib.orc_nyquist_stride.restype = i
            lib.orc_image.argtypes = [C.c_long, P, P, d, P]
            lib.orc_stack.argtypes = [i, i, i, P, i, i, i, i, P]
            lib.orc_energy.argtypes = [i, i, i, i, P, P, P]
            lib.orc_energy.restype = d
            lib.orc_splitmix64.argtypes = [u64, u64]
            lib.orc_splitmix64.restype = u64
            lib.orc_taper_g.argtypes = [d, i]
            lib.orc_taper_g.restype = d
            lib.orc_taper_h.argtypes = [d, i]
            lib.orc_taper_h.restype = d
            lib.orc_rbc_velocity.argtypes = [i, i, i, i, i, i, P, d, d, d, u64, i, P, P, P]
            lib.orc_rbc_velocity.restype = i
            lib.orc_coef.argtypes = [C.c_long, P, d, d, P, P]
            lib.orc_stencil_weights.argtypes = [P]
            lib.orc_fwi_grad.argtypes = [i, i, i, i, P, d, d, i, P, P, i, P, P, i, i, i, i, P]
            lib.orc_fwi_grad.restype = d
            lib.orc_misfit.argtypes = [i, i, i, i, P, d, i, P, P, i, P, P]
            lib.orc_misfit.restype = d
            _lib = lib
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dims(shape):
    """(ndim, NX, NY, NZ) from a dense array shape (NZ, NX) or (NZ, NY, NX)."""
    if len(shape) == 2:
        return 2, shape[1], 1, shape[0]
    return 3, shape[2], shape[1], shape[0]


def stencil_weights() -> np.ndarray:
    """8th-order central second-derivative weights c0..c4 (Section 4)."""
    out = np.zeros(5)
    _L().orc_stencil_weights(_p(out))
    return out


def lap8_point(p, x, y, z) -> float:
    """h^2 times the discrete Laplacian of Eq. 1 at one node (zero outside)."""
    p = _f64(p)
    nd, NX, NY, NZ = _dims(p.shape)
    return _L().orc_lap8_point(nd, NX, NY, NZ, _p(p), x, y, z)


def leapfrog(a, p_prev, p_cur):
    """One source-free leapfrog step of Eq. 1: 2 p - p_prev + a L8 p."""
    a, p_prev, p_cur = _f64(a), _f64(p_prev), _f64(p_cur)
    out = np.empty_like(p_cur)
    nd, NX, NY, NZ = _dims(a.shape)
    _L().orc_leapfrog(nd, NX, NY, NZ, _p(a), _p(p_prev), _p(p_cur), _p(out))
    return out


def model(a, h, nt, src, wavelet, rec, snaps=()):
    """Algorithm 1 for one shot.

    a: padded (v dt/h)^2, shape (NZ, NX) or (NZ, NY, NX); src: (x, y, z) padded
    node; rec: (nrec, 3) padded nodes; wavelet: nt samples (f[n] drives step
    n -> n+1).  Returns dict(seis=[nrec, nt+1], p_prev=p^{nt-1}, p_last=p^{nt},
    snaps=[len(snaps), ...] = p^n for n in snaps).
    """
    a = _f64(a)
    nd, NX, NY, NZ = _dims(a.shape)
    rec = _i32(np.asarray(rec).reshape(-1, 3))
    nrec = rec.shape[0]
    seis = np.zeros((nrec, nt + 1))
    pp, pl = np.zeros(a.shape), np.zeros(a.shape)
    sn = _i32(list(snaps))
    sv = np.zeros((len(sn),) + a.shape)
    rc = _L().orc_model(nd, NX, NY, NZ, _p(a), float(h), int(nt), _p(_i32(src)),
                        _p(_f64(wavelet)), nrec, _p(rec), _p(seis), _p(pp), _p(pl),
                        len(sn), _p(sn), _p(sv))
    if rc:
        raise ValueError("orc_model: bad argument")
    return dict(seis=seis, p_prev=pp, p_last=pl, snaps=sv)


def rtm_shot(a, h, nt, src, wavelet, rec, seis, nb, interior, reinject=True,
             rec_sign=REC_SIGN, snaps=(), top=None):
    """Algorithm 3 (RTM with wavefield reconstruction) for one shot.

    interior: (nx, ny, nz) box starting at padded node nb in x and y and at
    row top in z (default nb; 4 with a free surface).
    Returns dict(num, den) on the interior (shape (nz, nx) or (nz, ny, nx)) and
    optional snapshots pr/pb of p^R_n and pbar_n on the padded grid.
    """
    a = _f64(a)
    nd, NX, NY, NZ = _dims(a.shape)
    nx, ny, nz = interior
    ishape = (nz, nx) if nd == 2 else (nz, ny, nx)
    num, den = np.zeros(ishape), np.zeros(ishape)
    rec = _i32(np.asarray(rec).reshape(-1, 3))
    seis = _f64(seis)
    assert seis.shape == (rec.shape[0], nt + 1)
    sn = _i32(list(snaps))
    prs = np.zeros((len(sn),) + a.shape)
    pbs = np.zeros((len(sn),) + a.shape)
    rc = _L().orc_rtm_shot(nd, NX, NY, NZ, _p(a), float(h), int(nt), _p(_i32(src)),
                           _p(_f64(wavelet)), rec.shape[0], _p(rec), _p(seis),
                           int(bool(reinject)), float(rec_sign), int(nb), int(nb if top is None else top), int(nx),
                           int(ny if nd == 3 else 1), int(nz), _p(num), _p(den),
                           len(sn), _p(sn), _p(prs), _p(pbs))
    if rc:
        raise ValueError("orc_rtm_shot: bad argument")
    return dict(num=num, den=den, pr=prs, pb=pbs)


def nyquist_stride(dt, f_max, f_min=0.0) -> int:
    """Eq. 7: k = floor(dt_nyq / dt) with dt_nyq = 1 / (2 (f_max - f_min)); 0 on a bad argument."""
    return int(_L().orc_nyquist_stride(float(dt), float(f_max), float(f_min)))


def rtm_storage(a, h, nt, src, wavelet, rec, seis, nb, interior, stride, rec_sign=REC_SIGN,
                keep_store=False, top=None):
    """Algorithm 2 (RTM with wavefield storage) for one shot: the source
    wavefield is stored at levels 0, k, 2k, ... (k = stride) and the imaging
    integrals of Eq. 3 are accumulated at those levels only.

    Returns dict(num, den) on the interior and, with keep_store, the stored
    interior fields store[j] = p^{j k}."""
    a = _f64(a)
    nd, NX, NY, NZ = _dims(a.shape)
    nx, ny, nz = interior
    ishape = (nz, nx) if nd == 2 else (nz, ny, nx)
    num, den = np.zeros(ishape), np.zeros(ishape)
    rec = _i32(np.asarray(rec).reshape(-1, 3))
    seis = _f64(seis)
    assert seis.shape == (rec.shape[0], nt + 1)
    store = np.zeros((nt // stride + 1,) + ishape) if keep_store else None
    rc = _L().orc_rtm_storage(nd, NX, NY, NZ, _p(a), float(h), int(nt), _p(_i32(src)),
                              _p(_f64(wavelet)), rec.shape[0], _p(rec), _p(seis), float(rec_sign),
                              int(stride), int(nb), int(nb if top is None else top), int(nx),
                              int(ny if nd == 3 else 1), int(nz),
                              _p(num), _p(den), _p(store) if keep_store else None)
    if rc:
        raise ValueError("orc_rtm_storage: bad argument")
    out = dict(num=num, den=den)
    if keep_store:
        out["store"] = store
    return out


def image(num, den, eps_rel=1e-6):
    """Eq. 3 ratio formed once: I = num / (den + eps_rel * max(den))."""
    num, den = _f64(num), _f64(den)
    out = np.empty_like(num)
    _L().orc_image(num.size, _p(num), _p(den), float(eps_rel), _p(out))
    return out


def stack(survey, shot_img, off_x, off_y=0):
    """Algorithm 3 stacking: survey window at (off_x, off_y) += shot image (in place)."""
    assert survey.dtype == np.float64 and survey.flags.c_contiguous
    s = _f64(shot_img)
    if s.ndim == 2:
        nz, nx = s.shape
        ny, sy, sx = 1, 1, survey.shape[1]
    else:
        nz, ny, nx = s.shape
        sy, sx = survey.shape[1], survey.shape[2]
    _L().orc_stack(nx, ny, nz, _p(s), int(off_x), int(off_y), sx, sy, _p(survey))
    return survey


def energy(a, p0, p1) -> float:
    """Discrete energy of the undamped leapfrog between two consecutive levels."""
    a, p0, p1 = _f64(a), _f64(p0), _f64(p1)
    nd, NX, NY, NZ = _dims(a.shape)
    return _L().orc_energy(nd, NX, NY, NZ, _p(a), _p(p0), _p(p1))


def splitmix64(seed: int, j: int) -> int:
    """The j-th (j >= 1) output of the splitmix64 stream seeded with `seed`."""
    return int(_L().orc_splitmix64(C.c_uint64(seed), C.c_uint64(j)))


def taper_g(x, na):
    """Eq. 4."""
    return _L().orc_taper_g(float(x), int(na))


def taper_h(x, na):
    """Eq. 5."""
    return _L().orc_taper_h(float(x), int(na))


def rbc_velocity(v_int, nb, v_lo, v_hi, v_max, seed, mode=0, draws=False, free_surface=False):
    """Random-boundary padding of an interior velocity (Section 4.3, Eqs. 4-5).

    v_int: (nz, nx) or (nz, ny, nx).  Returns the padded velocity (and, with
    draws=True, the per-cell coefficient c and random velocity, NaN inside).
    free_surface: 4 zero-velocity rows on top instead of the random pad
    (Section 5's pressure-release surface); the interior then starts at row 4.
    """
    v = _f64(v_int)
    top = 4 if free_surface else nb
    if v.ndim == 2:
        nd, nz, ny, nx = 2, v.shape[0], 1, v.shape[1]
        shp = (nz + nb + top, nx + 2 * nb)
    else:
        nd, (nz, ny, nx) = 3, v.shape
        shp = (nz + nb + top, ny + 2 * nb, nx + 2 * nb)
    out = np.zeros(shp)
    c = np.zeros(shp) if draws else None
    vr = np.zeros(shp) if draws else None
    rc = _L().orc_rbc_velocity(nd, nx, ny, nz, int(nb), int(bool(free_surface)), _p(v), float(v_lo), float(v_hi),
                               float(v_max), C.c_uint64(seed), int(mode), _p(out), _p(c), _p(vr))
    if rc:
        raise ValueError("orc_rbc_velocity: bad argument")
    return (out, c, vr) if draws else out


def coef(v, dt, h):
    """a = (v dt / h)^2 in fp64 and its fp32 rounding."""
    v = _f64(v)
    a64 = np.empty_like(v)
    a32 = np.empty(v.shape, np.float32)
    _L().orc_coef(v.size, _p(v), float(dt), float(h), _p(a64), _p(a32))
    return a64, a32


def fwi_grad(a, h, dt, nt, src, wavelet, rec, d_obs, nb, interior):
    """Exact discrete adjoint gradient of J = 1/2 ||record - d_obs||^2 with
    respect to the interior velocity (random boundary fixed).  Returns (J, g)."""
    a = _f64(a)
    nd, NX, NY, NZ = _dims(a.shape)
    nx, ny, nz = interior
    g = np.zeros((nz, nx) if nd == 2 else (nz, ny, nx))
    rec = _i32(np.asarray(rec).reshape(-1, 3))
    J = _L().orc_fwi_grad(nd, NX, NY, NZ, _p(a), float(h), float(dt), int(nt), _p(_i32(src)),
                          _p(_f64(wavelet)), rec.shape[0], _p(rec), _p(_f64(d_obs)), int(nb), int(nx),
                          int(ny if nd == 3 else 1), int(nz), _p(g))
    return J, g


def misfit(a, h, nt, src, wavelet, rec, d_obs):
    """J = 1/2 sum (record - d_obs)^2 of Algorithm 1's record."""
    a = _f64(a)
    nd, NX, NY, NZ = _dims(a.shape)
    rec = _i32(np.asarray(rec).reshape(-1, 3))
    return _L().orc_misfit(nd, NX, NY, NZ, _p(a), float(h), int(nt), _p(_i32(src)), _p(_f64(wavelet)),
                           rec.shape[0], _p(rec), _p(_f64(d_obs)))
