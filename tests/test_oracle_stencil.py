"""Pins for the oracle's 8th-order Laplacian and leapfrog (Section 4: 8th order
in space, 2nd order in time).  Each check is a mathematical fact about the
discretisation, not a retyped formula."""
import math

import numpy as np
import pytest

import oracle


def _poly_field(shape, axis, m, x0, scale):
    idx = np.indices(shape)[axis].astype(np.float64)
    return ((idx - x0) / scale) ** m


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("m", range(0, 11))
def test_lap8_exact_on_polynomials_up_to_degree_9(ndim, m):
    # a central scheme of order 8 differentiates x^m exactly for m <= 9 and not for m = 10
    shape = (12, 12, 24) if ndim == 3 else (12, 24)
    axes = range(ndim)
    for axis in axes:
        p = _poly_field(shape, axis, m, x0=3.0, scale=4.0)
        pt = [6] * ndim
        pt[axis] = 13 if shape[axis] == 24 else 6
        coord = pt[axis]
        exact = m * (m - 1) * ((coord - 3.0) / 4.0) ** (m - 2) / 16.0 if m >= 2 else 0.0
        if ndim == 2:
            z, x = pt
            got = oracle.lap8_point(p, x, 0, z)
        else:
            z, y, x = pt
            got = oracle.lap8_point(p, x, y, z)
        if m <= 9:
            assert got == pytest.approx(exact, rel=1e-12, abs=1e-12)
        else:
            assert abs(got - exact) > 1e-9 * max(1.0, abs(exact))


def test_lap8_convergence_order_is_8():
    # error of h^-2 L8 sin(x) at the fixed point x = 6 falls as h^8
    errs = []
    for h in (0.6, 0.3, 0.15):
        j = int(round(6.0 / h))
        x = (np.arange(2 * j + 1) - 0.0) * h
        p = np.tile(np.sin(x), (9, 1))
        got = oracle.lap8_point(p, j, 0, 4) / h ** 2   # z-part is zero: rows are equal
        errs.append(abs(got + np.sin(6.0)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(7.7 < o < 8.3 for o in orders), orders


def test_symbol_and_stability_limit():
    # symbol of L8 at the Nyquist wavenumber decides the leapfrog limit:
    # v dt / h <= 2 / sqrt(d * |lambda_max|)
    c = oracle.stencil_weights()
    lam = c[0] + 2 * sum(c[k] * math.cos(k * math.pi) for k in range(1, 5))
    assert lam == pytest.approx(-6.501587301587, rel=1e-12)
    for d, limit in ((2, 0.5546), (3, 0.4529)):
        assert 2 / math.sqrt(d * -lam) == pytest.approx(limit, abs=1e-4)


@pytest.mark.parametrize("courant,stable", [(0.55, True), (0.56, False)])
def test_leapfrog_stability_limit_2d(courant, stable):
    # the 2-D scheme stays bounded just below v dt/h = 0.5546 and blows up just above
    rng = np.random.default_rng(0)
    a = np.full((40, 40), courant ** 2)
    p0 = rng.standard_normal(a.shape)
    p1 = p0.copy()
    for _ in range(400):
        p0, p1 = p1, oracle.leapfrog(a, p0, p1)
    grown = np.abs(p1).max() > 1e3
    assert grown != stable


def _lam(c, k):
    return c[0] + 2 * sum(c[m] * np.cos(m * k) for m in range(1, 5))


@pytest.mark.parametrize("ndim", [2, 3])
def test_discrete_plane_wave_is_exact(ndim):
    # cos(k.x - w n) solves the recursion exactly when 2 - 2 cos w = -a sum_axes lambda(k_axis)
    c = oracle.stencil_weights()
    a0 = 0.16
    ks = (0.31, 0.47, 0.23)[:ndim]
    lam = sum(_lam(c, k) for k in ks)
    w = math.acos(1 + a0 * lam / 2)
    n0 = 40 if ndim == 3 else 100
    shape = (n0,) * ndim
    grids = np.indices(shape).astype(np.float64)  # z, (y), x
    phase = sum(k * g for k, g in zip(ks, grids[::-1]))
    a = np.full(shape, a0)
    p_prev, p_cur = np.cos(phase + w), np.cos(phase)   # n = -1, 0
    nsteps = 3
    for n in range(1, nsteps + 1):
        p_prev, p_cur = p_cur, oracle.leapfrog(a, p_prev, p_cur)
    exact = np.cos(phase - w * nsteps)
    m = 4 * nsteps + 4     # outside the domain of dependence of the truncation
    core = tuple(slice(m, s - m) for s in shape)
    assert np.abs(p_cur[core] - exact[core]).max() < 1e-12


def test_energy_is_conserved_by_the_source_free_recursion():
    rng = np.random.default_rng(3)
    a = rng.uniform(0.05, 0.25, (30, 26))
    p0 = rng.standard_normal(a.shape)
    p1 = p0 + 0.01 * rng.standard_normal(a.shape)
    e0 = oracle.energy(a, p0, p1)
    for _ in range(300):
        p0, p1 = p1, oracle.leapfrog(a, p0, p1)
    assert oracle.energy(a, p0, p1) == pytest.approx(e0, rel=1e-12)


def test_energy_catches_an_asymmetric_operator():
    # a perturbed (non-symmetric) stencil must break conservation: the pin has teeth
    rng = np.random.default_rng(4)
    a = rng.uniform(0.05, 0.25, (30, 26))
    p0 = rng.standard_normal(a.shape)
    p1 = p0.copy()
    e0 = oracle.energy(a, p0, p1)
    for _ in range(100):
        nxt = oracle.leapfrog(a, p0, p1)
        nxt[:, 1:] += 1e-3 * a[:, 1:] * p1[:, :-1]   # one-sided extra term
        p0, p1 = p1, nxt
    assert abs(oracle.energy(a, p0, p1) - e0) > 1e-8 * abs(e0)
