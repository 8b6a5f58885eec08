"""Pins for the oracle's free-surface option (Section 5: the top of the grid
carries half the stencil length, 4 rows, of zero pressure instead of the
random pad):

* the grid arithmetic the paper prints (737 x 240 + 50 -> 837 x 294);
* the random pad of the sides and the bottom keeps the tapers of Eqs. 4-5
  with the distance measured from the sides and the bottom only;
* physics: a pressure-release surface reflects with coefficient -1, so a
  shallow source and receiver see the direct wave minus its mirror image
  (the analytic 3-D Green's function of the source and of its image about
  the last zero row);
* brute force of Algorithms 1/3 with the interior window starting at row 4,
  and exact time reversibility through the random sides.
"""
import json
import math
import os

import numpy as np

import oracle
import workloads as W
from test_oracle_green import V, green_3d, ricker
from test_oracle_rtm import dense_pipeline

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_padded_grid_of_section_5():
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["padded_grid_2d"]
    nx, nz = g["interior"]
    v = np.full((nz, nx), 2000.0)
    vp = oracle.rbc_velocity(v, g["na"], 1500.0, 4500.0, 4500.0, 1, free_surface=True)
    assert list(vp.shape[::-1]) == g["padded_printed"]
    assert np.all(vp[: g["top_pad"]] == 0.0)                       # the zero-pressure rows
    top, nb = g["top_pad"], g["na"]
    np.testing.assert_array_equal(vp[top:top + nz, nb:nb + nx], v)  # interior untouched
    assert np.all(vp[top:, :nb] > 0) and np.all(vp[top + nz:, :] > 0)


def test_side_pad_distance_ignores_the_surface():
    nb, nx, nz = 12, 30, 20
    v = np.full((nz, nx), 2500.0)
    _, c, vr = oracle.rbc_velocity(v, nb, 1500.0, 4500.0, 4500.0, 5, draws=True, free_surface=True)
    for i in range(1, nb + 1):                     # left pad, first interior row: distance = i
        col = nb - i
        ci = c[4, col]
        g, h = oracle.taper_g(i, nb), oracle.taper_h(i, nb)
        assert min(g, h) - 1e-12 <= ci <= max(g, h) + 1e-12
    # in the rows next to the surface the distance is the column distance, not
    # a distance to the (absent) top pad: compare with the row 20 rows lower
    lo_g, lo_h = oracle.taper_g(nb, nb), oracle.taper_h(nb, nb)
    assert min(lo_g, lo_h) - 1e-12 <= c[4, 0] <= max(lo_g, lo_h) + 1e-12
    assert np.isnan(c[4:4 + nz, nb:nb + nx]).all() and np.isnan(c[:4]).all()


def _ghost_error(z_surface_rows):
    h, dt, n, T = 10.0, 1e-3, 61, 0.25
    nt = int(round(T / dt))
    a = np.full((n, n, n), (V * dt / h) ** 2)
    a[:4] = 0.0                                    # the four zero-pressure rows
    c, zs = n // 2, 6                              # source 2 cells below the first interior row
    src = np.array([c, c, zs], np.int32)
    dists = [100.0, 150.0]
    rec = np.array([[c + int(round(d / h)), c, zs] for d in dists], np.int32)
    wav = np.array([ricker(k * dt) for k in range(nt)])
    seis = oracle.model(a, h, nt, src, wav, rec)["seis"]
    errs = []
    for i, d in enumerate(dists):
        r2 = math.hypot(d, 2 * (zs - z_surface_rows) * h)   # the image source
        ex = np.array([green_3d(d, k * dt) - green_3d(r2, k * dt) for k in range(nt + 1)])
        errs.append(np.linalg.norm(seis[i] - ex) / np.linalg.norm(ex))
    return max(errs)


def test_pressure_release_surface_makes_a_negative_ghost():
    assert _ghost_error(3.0) < 0.08                # surface at the last zero row
    assert _ghost_error(3.5) > 0.2                 # half a cell off is clearly worse
    assert _ghost_error(6.0 + 1e6) > 0.5           # no ghost at all (mirror far away) fails


def _fs_case(ndim, seed):
    rng = np.random.default_rng(seed)
    if ndim == 2:
        nx, ny, nz, nb = 8, 1, 6, 3
        shape = (nz + nb + 4, nx + 2 * nb)
        src = np.array([nb + 4, 0, 5], np.int32)
        rec = np.array([[nb + i, 0, 4] for i in range(nx)], np.int32)
    else:
        nx, ny, nz, nb = 5, 4, 4, 3
        shape = (nz + nb + 4, ny + 2 * nb, nx + 2 * nb)
        src = np.array([nb + 2, nb + 1, 5], np.int32)
        rec = np.array([[nb + i, nb + j, 4] for j in range(ny) for i in range(nx)], np.int32)
    a_true = rng.uniform(0.05, 0.2, shape)
    a_mig = rng.uniform(0.05, 0.2, shape)
    a_true[:4] = 0.0
    a_mig[:4] = 0.0
    return (nx, ny, nz), nb, src, rec, a_true, a_mig, rng


def test_bruteforce_rtm_with_free_surface():
    for ndim in (2, 3):
        interior, nb, src, rec, a_true, a_mig, rng = _fs_case(ndim, 30 + ndim)
        h, nt = 7.0, 30
        wav = rng.standard_normal(nt)
        seis_d, num_d, den_d = dense_pipeline(a_true, a_mig, h, nt, src, wav, rec, nb, interior)
        # dense_pipeline's window starts at nb on every axis; recompute it at row 4
        shape = a_true.shape
        full = dense_pipeline(a_true, a_mig, h, nt, src, wav, rec, 0,
                              (shape[-1], shape[1] if ndim == 3 else 1, shape[0]))
        nx, ny, nz = interior
        win = ((slice(4, 4 + nz), slice(nb, nb + nx)) if ndim == 2 else
               (slice(4, 4 + nz), slice(nb, nb + ny), slice(nb, nb + nx)))
        num_d, den_d = full[1][win], full[2][win]
        seis = oracle.model(a_true, h, nt, src, wav, rec)["seis"]
        np.testing.assert_allclose(seis, seis_d, rtol=1e-12, atol=1e-12 * np.abs(seis_d).max())
        r = oracle.rtm_shot(a_mig, h, nt, src, wav, rec, seis, nb, interior, top=4)
        np.testing.assert_allclose(r["num"], num_d, rtol=1e-10, atol=1e-11 * np.abs(num_d).max())
        np.testing.assert_allclose(r["den"], den_d, rtol=1e-10, atol=1e-11 * np.abs(den_d).max())
        st = oracle.rtm_storage(a_mig, h, nt, src, wav, rec, seis, nb, interior, 1, top=4)
        np.testing.assert_allclose(st["num"], num_d, rtol=1e-10, atol=1e-11 * np.abs(num_d).max())


def test_reversibility_with_free_surface():
    w = W.scaled(W.SMALL_2D, nx=80, nz=60, nb=20, nt=500, name="fsrev")
    vp = oracle.rbc_velocity(np.full((w.nz, w.nx), 2000.0), w.nb, w.v_lo, w.v_hi, w.v_max, 2, free_surface=True)
    a = oracle.coef(vp, w.dt, w.h)[1].astype(np.float64)
    src = np.array([w.nb + w.nx // 2, 0, 4 + 2], np.int32)
    wav = W.ricker(w.nt, w.dt, w.f_peak)
    snaps = [0, w.nt // 4, w.nt // 2, w.nt]
    none = np.zeros((0, 3), np.int32)
    fwd = oracle.model(a, w.h, w.nt, src, wav, none, snaps=snaps)["snaps"]
    r = oracle.rtm_shot(a, w.h, w.nt, src, wav, none, np.zeros((0, w.nt + 1)), w.nb, (w.nx, 1, w.nz),
                        snaps=snaps, top=4)
    ref = np.linalg.norm(fwd[2])
    for k in range(len(snaps)):
        assert np.linalg.norm(r["pr"][k] - fwd[k]) <= 1e-10 * ref
    assert np.all(fwd[:, :4] == 0.0)               # the surface rows never move
