"""Pin the oracle's FWI gradient (exact discrete adjoint of Algorithm 1's
recursion, random boundary held fixed) against central finite differences of
its own misfit J = 1/2 ||record - d_obs||^2 at 20 seeded interior points."""
import numpy as np
import pytest

import oracle
import workloads as W


def _case(seed=0):
    w = W.scaled(W.SMALL_2D, nx=40, nz=30, nb=8, nt=250, name="fwi_pin")
    vt = W.three_layers(w.nx, w.nz, (10, 20))
    vt[12:18, 15:25] *= 1.1
    v0 = W.smooth_slowness(vt, 3.0)
    src, rec = W.source_at(w, 20), W.surface_line(w, step=2)
    wav = W.ricker(w.nt, w.dt, w.f_peak)
    return w, vt, v0, src, rec, wav


def _a(w, v):
    return oracle.coef(oracle.rbc_velocity(v, w.nb, 1500, 4500, 4000, 1), w.dt, w.h)[0]


def test_fwi_gradient_matches_finite_differences():
    w, vt, v0, src, rec, wav = _case()
    dobs = oracle.model(_a(w, vt), w.h, w.nt, src, wav, rec)["seis"]
    J, g = oracle.fwi_grad(_a(w, v0), w.h, w.dt, w.nt, src, wav, rec, dobs, w.nb, (w.nx, 1, w.nz))
    assert J == pytest.approx(oracle.misfit(_a(w, v0), w.h, w.nt, src, wav, rec, dobs), rel=1e-12)
    rng = np.random.default_rng(20)
    # interior points off the edge cells (edge cells also set the boundary's v_edge)
    pts = [(rng.integers(1, w.nz - 1), rng.integers(1, w.nx - 1)) for _ in range(20)]
    gmax = np.abs(g).max()
    for iz, ix in pts:
        d = 1e-4 * v0[iz, ix]
        vp, vm = v0.copy(), v0.copy()
        vp[iz, ix] += d
        vm[iz, ix] -= d
        fd = (oracle.misfit(_a(w, vp), w.h, w.nt, src, wav, rec, dobs)
              - oracle.misfit(_a(w, vm), w.h, w.nt, src, wav, rec, dobs)) / (2 * d)
        assert abs(g[iz, ix] - fd) <= 1e-6 * abs(fd) + 1e-6 * gmax, (iz, ix, g[iz, ix], fd)


def test_fwi_gradient_vanishes_at_the_true_model_and_points_downhill():
    w, vt, v0, src, rec, wav = _case()
    dobs = oracle.model(_a(w, vt), w.h, w.nt, src, wav, rec)["seis"]
    J0, g0 = oracle.fwi_grad(_a(w, vt), w.h, w.dt, w.nt, src, wav, rec, dobs, w.nb, (w.nx, 1, w.nz))
    assert J0 == 0.0 and np.all(g0 == 0.0)
    J, g = oracle.fwi_grad(_a(w, v0), w.h, w.dt, w.nt, src, wav, rec, dobs, w.nb, (w.nx, 1, w.nz))
    step = 20.0 / np.abs(g).max()          # at most 20 m/s per cell
    J1 = oracle.misfit(_a(w, v0 - step * g), w.h, w.nt, src, wav, rec, dobs)
    assert J1 < J
