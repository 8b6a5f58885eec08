"""Pin the oracle's modeling loop (Algorithm 1 with the point source of Eq. 1)
to the analytic Green's function of the homogeneous acoustic wave equation.

For  lap p - p_tt / v^2 = f(t) delta(r):
  3-D:  p = -f(t - r/v) / (4 pi r)
  2-D:  p = -(1 / 2 pi) int_{r/v}^inf f(t - s) / sqrt(s^2 - r^2/v^2) ds
            = -(1 / 2 pi) int_0^inf f(t - (r/v) cosh u) du
The medium is 2000 m/s, the value of the paper's Figure 1.  Traces are
compared before any boundary reflection arrives; the discrete error is
second order in (h, dt) refined together.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle

V = 2000.0
F = 15.0
T0 = 1.5 / F


def ricker(t):
    x = (math.pi * F * (t - T0)) ** 2
    return (1 - 2 * x) * math.exp(-x)


def green_2d(r, t):
    if t <= r / V:
        return 0.0
    umax = math.acosh((t + 1.0) / (r / V))
    val, _ = quad(lambda u: ricker(t - (r / V) * math.cosh(u)), 0, umax, limit=400,
                  epsabs=1e-12)
    return -val / (2 * math.pi)


def green_3d(r, t):
    return -ricker(t - r / V) / (4 * math.pi * r)


def _traces(ndim, h, dt, n, T, dists_m):
    nt = int(round(T / dt))
    shape = (n,) * ndim
    a = np.full(shape, (V * dt / h) ** 2)
    c = n // 2
    src = np.array([c, c if ndim == 3 else 0, c], np.int32)
    rec = np.array([[c + int(round(d / h)), c if ndim == 3 else 0, c] for d in dists_m], np.int32)
    wav = np.array([ricker(k * dt) for k in range(nt)])
    seis = oracle.model(a, h, nt, src, wav, rec)["seis"]
    g = green_2d if ndim == 2 else green_3d
    errs = []
    for i, d in enumerate(dists_m):
        ex = np.array([g(d, k * dt) for k in range(nt + 1)])
        errs.append(np.linalg.norm(seis[i] - ex) / np.linalg.norm(ex))
    return np.array(errs)


def test_green_2d_and_second_order_refinement():
    coarse = _traces(2, 10.0, 1e-3, 201, 0.55, (200.0, 400.0))
    fine = _traces(2, 5.0, 5e-4, 401, 0.55, (200.0, 400.0))
    assert np.all(coarse < 2e-2), coarse
    assert np.all(coarse / fine > 3.0), coarse / fine


def test_green_3d_and_second_order_refinement():
    coarse = _traces(3, 10.0, 1e-3, 81, 0.3, (100.0, 160.0))
    fine = _traces(3, 5.0, 5e-4, 161, 0.3, (100.0, 160.0))
    assert np.all(coarse < 1e-2), coarse
    assert np.all(coarse / fine > 3.0), coarse / fine


def test_green_catches_a_wrong_source_scale():
    # the same comparison fails by far if the source strength were off by h (3-D)
    h, dt, n = 10.0, 1e-3, 81
    nt = 300
    a = np.full((n, n, n), (V * dt / h) ** 2)
    c = n // 2
    wav = np.array([ricker(k * dt) for k in range(nt)]) * h   # planted mistake
    rec = np.array([[c + 10, c, c]], np.int32)
    seis = oracle.model(a, h, nt, np.array([c, c, c], np.int32), wav, rec)["seis"][0]
    ex = np.array([green_3d(100.0, k * dt) for k in range(nt + 1)])
    assert np.linalg.norm(seis - ex) / np.linalg.norm(ex) > 1.0
