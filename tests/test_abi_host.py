"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/rbc.h declares, and rejects bad arguments before
touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as G
    b = G._builder()
    b.build()
    return C.CDLL(b.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n


def test_binding_exposes_the_same_names():
    import paper_2204_03380_gb300 as R
    assert sorted(R.EXPORTED) == _declared()


def test_bad_arguments_are_rejected_on_the_host():
    import paper_2204_03380_gb300 as R
    lib = R._native._lib
    g = R.make_grid(2, 10, 1, 10, 5, 10.0, 1e-3, 10)
    out = C.c_void_p()
    assert lib.rbc_create(None, None, C.byref(out)) == 1
    assert "NULL" in R.rbc_last_error()
    bad = R.make_grid(4, 10, 1, 10, 5, 10.0, 1e-3, 10)
    assert lib.rbc_create(C.byref(bad), C.c_void_p(16), C.byref(out)) == 1
    fs = R.make_grid(2, 10, 1, 10, 5, 10.0, 1e-3, 10, free_surface=2)
    assert lib.rbc_create(C.byref(fs), C.c_void_p(16), C.byref(out)) == 1
    assert R.make_grid(2, 10, 1, 10, 5, 10.0, 1e-3, 10, free_surface=1).padded == (10 + 5 + 4, 20)
    nb1 = R.make_grid(2, 10, 1, 10, 1, 10.0, 1e-3, 10)
    assert lib.rbc_build_velocity(C.byref(nb1), C.c_void_p(16), 1.0, 2.0, 2.0, 0, 0, None,
                                  C.c_void_p(16), None) == 1
    assert lib.rbc_build_velocity(C.byref(g), C.c_void_p(16), 1.0, 2.0, 2.0, 0, 2, None,
                                  C.c_void_p(16), None) == 1
    assert lib.rbc_build_velocity(C.byref(g), C.c_void_p(16), 3.0, 2.0, 2.0, 0, 0, None,
                                  C.c_void_p(16), None) == 1
    # image stack window checks
    shot = R.make_grid(2, 10, 1, 8, 5, 10.0, 1e-3, 10)
    survey = R.make_grid(2, 15, 1, 8, 5, 10.0, 1e-3, 10)
    p = C.c_void_p(16)
    assert lib.rbc_image_stack(C.byref(shot), p, p, 1e-6, 6, 0, C.byref(survey), p, None) == 1
    assert lib.rbc_image_stack(C.byref(shot), p, p, 1e-6, 0, 1, C.byref(survey), p, None) == 1
    other = R.make_grid(2, 15, 1, 9, 5, 10.0, 1e-3, 10)
    assert lib.rbc_image_stack(C.byref(shot), p, p, 1e-6, 0, 0, C.byref(other), p, None) == 1
    assert lib.rbc_model(None, None, None, 0, None, None, None) == 1
    assert lib.rbc_set_snapshots(None, 0, None, None, None, None) == 1
    assert lib.rbc_set_coef(None, C.c_void_p(16), 1, None) == 1
    # the other entry points' argument checks come before any device work
    assert lib.rbc_rtm_shot(None, None, None, 0, None, None, 1, None, None, None) == 1
    assert lib.rbc_rtm_storage(None, None, None, 0, None, None, 1, None, C.c_longlong(0), 0, None, None, None) == 1
    assert lib.rbc_fwi_forward(None, None, None, 1, None, None, None, None, None, None) == 1
    assert lib.rbc_fwi_backward(None, None, None, 1, None, None, None, None, None) == 1
    assert lib.rbc_get_panels(None, None, None, None) == 1
    assert lib.rbc_phase_timing(None, 1, None) == 1
    assert lib.rbc_inject_fault(None, 2) == 1          # unknown mode
    assert lib.rbc_inject_fault(None, 1) == 0          # arms the next 3-D rbc_model_static call
    assert lib.rbc_inject_fault(None, 0) == 0          # and clears it again
    out_b = C.c_void_p()
    nx1 = (C.c_int * 1)(10)
    assert lib.rbc_batch_create(C.byref(g), 0, nx1, None, C.byref(out_b)) == 1
    g3 = R.make_grid(3, 10, 10, 10, 5, 10.0, 1e-3, 10)
    ptrs = (C.c_void_p * 1)(16)
    assert lib.rbc_batch_create(C.byref(g3), 1, nx1, ptrs, C.byref(out_b)) == 6   # batches are 2-D
    assert lib.rbc_batch_create(C.byref(R.make_grid(2, 10, 1, 10, 5, 10.0, 1e-3, 10, free_surface=1)), 1, nx1,
                                ptrs, C.byref(out_b)) == 1
    assert lib.rbc_batch_rtm(None, None, None, 1, C.c_float(1e-6), None, 10, None) == 1
    assert lib.rbc_batch_timing(None, 0, None) == 1
    assert lib.rbc_batch_info(None, None) == 1
    p16 = C.c_void_p(16)
    assert lib.rbc_cnn_forward(None, 1, 8, 8, p16, p16, p16, None) == 1
    assert lib.rbc_cnn_forward(p16, 0, 8, 8, p16, p16, p16, None) == 1
    assert lib.rbc_cnn_infer(p16, 1, 8, 8, None, p16, p16, None) == 1
    assert lib.rbc_cnn_infer(p16, 1, 8, 0, p16, p16, p16, None) == 1
    assert lib.rbc_cnn_backward(p16, 1, 0, 8, p16, p16, p16, None) == 1
    assert lib.rbc_cnn_mse(p16, p16, C.c_longlong(0), None, p16, None) == 1
    assert lib.rbc_cnn_adam(p16, p16, p16, p16, C.c_float(1e-3), C.c_float(0.9), C.c_float(0.999),
                            C.c_float(1e-8), 0, None) == 1
    assert lib.rbc_model_static(None, None, None, None, 0, None, None, None) == 1
    # grids whose plane (pitch x rows) or buffer exceeds 32-bit offsets are
    # refused on the host, before any device work, by the context and the
    # static path alike (the extents are formed in 64-bit first)
    src = (C.c_int * 3)(5, 5, 1)
    for big in (R.make_grid(3, 60000, 60000, 1, 2, 10.0, 1e-3, 10), R.make_grid(2, 2000000000, 1, 4, 2, 10.0, 1e-3, 10),
                R.make_grid(3, 3000, 3000, 300, 2, 10.0, 1e-3, 10)):
        assert lib.rbc_model_static(C.byref(big), p16, src, p16, 0, None, None, None) == 1
        out_c = C.c_void_p()
        assert lib.rbc_create(C.byref(big), p16, C.byref(out_c)) == 1 and not out_c.value


def test_nyquist_stride_and_storage_size_on_the_host():
    # host-only entry points: Eq. 7 against the oracle's independent version
    # and the paper's 5 ms step, and the store size formula
    import json
    import oracle
    import paper_2204_03380_gb300 as R
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    n = g["nyquist_step_2d"]
    assert R.rbc_nyquist_stride(n["dt"], n["f_max"], n["f_min"]) == n["stride"]
    for dt, fmax, fmin in [(0.001, 37.5, 0.0), (0.0004, 62.5, 0.0), (0.001, 40.0, 10.0), (0.004, 1000.0, 0.0)]:
        assert R.rbc_nyquist_stride(dt, fmax, fmin) == oracle.nyquist_stride(dt, fmax, fmin)
    with pytest.raises(R.RBCError):
        R.rbc_nyquist_stride(0.001, 10.0, 20.0)
    grid = R.make_grid(3, 10, 7, 5, 4, 10.0, 1e-3, 23)
    assert R.rbc_storage_bytes(grid, 4) == 4 * 10 * 7 * 5 * (23 // 4 + 1)
    grid = R.make_grid(2, 10, 1, 5, 4, 10.0, 1e-3, 24)
    assert R.rbc_storage_bytes(grid, 4) == 4 * 10 * 5 * 7
    with pytest.raises(R.RBCError):
        R.rbc_storage_bytes(grid, 0)


def test_paper_receiver_grid_of_eqs_8_9():
    # host geometry: the 320 x 320 receivers of Eqs. 8-9 on the 25 m grid of
    # the 10 km model land on consecutive nodes 40 .. 359 (1012.5 m rounds to
    # node 41 with halves rounded up) in both axes
    import json
    import numpy as np
    import workloads as W
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["receivers_3d"]
    n = int(g["extent_m"] / g["h"]) + 1
    w = W.scaled(W.SHOT_3D, nx=n, ny=n, nz=20, nb=5, name="hpc4e")
    w = W.dataclasses.replace(w, h=g["h"])
    rec = W.receiver_grid_m(w, g["start_m"], g["spacing_m"], g["count"], top=4)
    assert rec.shape == (g["count"] ** 2, 3)
    xs = np.unique(rec[:, 0]) - w.nb
    assert xs[0] == 41 and xs[-1] == 360 and np.all(np.diff(xs) == 1)
    assert np.all(rec[:, 2] == 5)
