"""Pins for the random boundary (Section 4.3, Eqs. 4-5) and its generator."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_first_output():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    assert oracle.splitmix64(g["seed"], g["j"]) == int(g["value_hex"], 16)


def test_splitmix64_uniform_bits():
    vals = np.array([oracle.splitmix64(12345, j) for j in range(1, 20001)], dtype=np.uint64)
    u = (vals >> np.uint64(11)).astype(np.float64) / 2.0 ** 53
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    bits = np.unpackbits(vals.view(np.uint8)).reshape(-1, 64).mean(0)
    assert np.all(np.abs(bits - 0.5) < 0.02)


def test_tapers_match_the_printed_values():
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))
    for x, na, val in g["taper_g"]["cases"]:
        assert oracle.taper_g(x, na) == pytest.approx(val, abs=1e-15)
    for x, na, val in g["taper_h"]["cases"]:
        assert oracle.taper_h(x, na) == pytest.approx(val, rel=1e-12, abs=0)
    # h lies below g on the whole pad (the coefficient interval h <= c <= g)
    for na in (20, 50, 60):
        xs = np.arange(1, na)
        assert all(oracle.taper_h(x, na) <= oracle.taper_g(x, na) + 1e-15 for x in xs)


@pytest.mark.parametrize("ndim", [2, 3])
def test_rbc_draws_and_bounds(ndim):
    nb = 12
    if ndim == 2:
        v = W.three_layers(40, 30, (10, 20))
    else:
        v = np.full((10, 12, 14), 2500.0)
        v[5:] = 3500.0
    vp, c, vr = oracle.rbc_velocity(v, nb, 1500.0, 4500.0, 3500.0, seed=9, draws=True)
    pad = np.isfinite(c)
    inner = (slice(nb, -nb),) * ndim
    assert not pad[inner].any() and pad.sum() == vp.size - v.size
    np.testing.assert_array_equal(vp[inner], v)                 # interior untouched
    # distance into the pad (max norm) and the coefficient interval of Eqs. 4-5
    idx = np.indices(vp.shape)
    dist = np.zeros(vp.shape, np.int64)
    for ax, n in enumerate(v.shape):
        q = idx[ax]
        dist = np.maximum(dist, np.where(q < nb, nb - q, np.where(q >= nb + n, q - (nb + n - 1), 0)))
    for i in range(1, nb + 1):
        sel = dist == i
        lo = min(oracle.taper_h(i, nb), oracle.taper_g(i, nb))
        hi = max(oracle.taper_h(i, nb), oracle.taper_g(i, nb))
        assert np.all(c[sel] >= lo - 1e-15) and np.all(c[sel] <= hi + 1e-15)
        if hi - lo > 0.05 and sel.sum() > 200:
            assert stats.kstest((c[sel] - lo) / (hi - lo), "uniform").pvalue > 1e-4
    assert np.all(c[dist == 1] == 1.0)           # g(1) = h(1) = 1: continuous at the edge
    assert np.all(vr[pad] >= 1500.0) and np.all(vr[pad] < 4500.0)
    assert vp.max() <= 3500.0 and vp.min() >= 1500.0 - 1e-9   # capped: stability kept


def test_rbc_is_deterministic_and_seeds_decorrelate():
    v = W.three_layers(50, 40, (10, 20))
    a = oracle.rbc_velocity(v, 15, 1500, 4500, 3500, seed=1)
    b = oracle.rbc_velocity(v, 15, 1500, 4500, 3500, seed=1)
    c = oracle.rbc_velocity(v, 15, 1500, 4500, 3500, seed=2)
    np.testing.assert_array_equal(a, b)
    outer = np.zeros(a.shape, bool)
    outer[:5] = outer[-5:] = True
    outer[:, :5] = outer[:, -5:] = True
    assert abs(np.corrcoef(a[outer], c[outer])[0, 1]) < 0.1


def test_rbc_literal_mode():
    v = np.full((20, 20), 3000.0)
    vp, c, vr = oracle.rbc_velocity(v, 8, 1500, 4500, 4000, seed=3, mode=1, draws=True)
    pad = np.isfinite(c)
    np.testing.assert_allclose(vp[pad], np.minimum(np.maximum(c[pad] * vr[pad], 1500), 4000))


@pytest.mark.parametrize("w", [W.SMALL_2D, W.SURVEY_2D, W.SHOT_3D], ids=lambda w: w.name)
def test_workload_presets_are_stable(w):
    # the cap v_max keeps v dt / h below the stability limit of the scheme
    c = oracle.stencil_weights()
    lam = -(c[0] + 2 * sum(c[k] * (-1) ** k for k in range(1, 5)))
    courant = w.v_max * w.dt / w.h
    assert courant ** 2 * w.ndim * lam < 4.0


def test_two_panel_storage_matches_table_4():
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["two_panel_storage_3d"]
    nbytes = g["panels"] * int(np.prod(g["grid"])) * g["bytes_per_value"]
    assert nbytes / 2 ** 30 == pytest.approx(g["gb_printed"], abs=5e-4)


def test_padded_grid_arithmetic_of_section_5():
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["padded_grid_2d"]
    nx, nz = g["interior"]
    assert [nx + 2 * g["na"], nz + g["na"] + g["top_pad"]] == g["padded_printed"]
