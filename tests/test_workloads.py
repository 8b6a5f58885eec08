"""The synthetic input recipes: the presets and generators hold the sizes,
geometry, value ranges and stability margins stated for each workload, and
they are deterministic (every input of the tests and the bench is seeded)."""
import numpy as np
import pytest

import workloads as W

# the scheme's stability limit on v dt / h: a * ndim * 6.5016 < 4 with the 8th-order symbol
LIMIT = {2: np.sqrt(4.0 / (2 * 6.501587301587302)), 3: np.sqrt(4.0 / (3 * 6.501587301587302))}


@pytest.mark.parametrize("w", [W.SMALL_2D, W.SURVEY_2D, W.SHOT_3D, W.BATCH_2D, W.FWI_2D],
                         ids=lambda w: w.name)
def test_presets_are_stable_with_their_boundary_velocities(w):
    # the random boundary is capped at v_max, and v_max bounds every interior model
    assert w.v_lo < w.v_hi and w.v_max <= w.v_hi
    assert w.v_max * w.dt / w.h < LIMIT[w.ndim]


def test_survey_recipe():
    w = W.SURVEY_2D
    assert (w.nx, w.nz, w.nb, w.h, w.dt, w.nt, w.f_peak, w.nshots) == (2301, 751, 60, 4.0, 0.4e-3, 12500, 25.0, 240)
    assert w.padded == (871, 2421)
    inp = W.survey_2d_inputs(w)
    v = inp["v_true"]
    assert v.shape == (751, 2301) and v.min() >= 1500.0 - 1e-3 and v.max() <= 5500.0 + 1e-3
    # migration model: smoothed slowness, so smaller jumps between neighbours
    assert np.abs(np.diff(inp["v_mig"], axis=0)).max() < np.abs(np.diff(v, axis=0)).max()
    shots = inp["shots"]
    assert len(shots) == 240 and np.all(np.diff(shots) > 0) and shots.min() >= 0 and shots.max() < w.nx
    rec = inp["rec"]
    assert rec.shape == (460, 3) and np.all(np.diff(rec[:, 0]) == 5)
    assert np.all(rec[:, 2] == w.nb + 1) and rec[:, 0].max() < w.nb + w.nx


def test_3d_recipe():
    w = W.SHOT_3D
    assert w.padded == (380, 580, 580)
    inp = W.shot_3d_inputs(w)
    assert inp["v"].shape == (300, 500, 500)
    assert inp["v"].min() >= 1500.0 - 1e-3 and inp["v"].max() <= 4500.0 + 1e-3
    assert len(inp["rec"]) == 250 * 250
    assert list(inp["src"]) == [250 + 40, 250 + 40, 41]


def test_batch_recipe():
    w = W.BATCH_2D
    inp = W.batch_2d_inputs(w)
    shots = inp["shots"]
    assert len(shots) == 64
    widths = np.array([s["width"] for s in shots])
    assert widths.min() >= 400 and widths.max() <= 1200 and len(set(widths.tolist())) > 32
    for s in shots:
        assert 0 <= s["off_x"] and s["off_x"] + s["width"] <= w.nx
        # source at the window centre, receivers every 2 columns, all at depth 1 in the shot's frame
        assert s["src"][0] == s["width"] // 2 + w.nb and s["src"][2] == w.nb + 1
        assert np.all(np.diff(s["rec"][:, 0]) == 2) and s["rec"][:, 0].max() < s["width"] + w.nb
    v = inp["v_true"]
    assert v.shape == (600, 4000) and v.min() >= w.v_lo - 1e-3 and v.max() <= w.v_max + 1e-3


def test_fwi_recipe():
    w = W.FWI_2D
    inp = W.fwi_2d_inputs(w)
    vt, v0 = inp["v_true"], inp["v0"]
    assert vt.shape == v0.shape == (300, 300)
    # +10 % anomaly at the centre, inside the 2500 m/s layer
    assert vt[150, 150] == pytest.approx(2750.0, rel=1e-6)
    assert vt[0, 0] == 1500.0 and vt[-1, -1] == pytest.approx(3500.0, rel=1e-3)
    assert len(inp["srcs"]) == 4 and len(inp["rec"]) == 150
    assert np.abs(v0 - vt).max() > 100.0       # the starting model differs from the truth


def test_generators_are_deterministic():
    a, b = W.batch_2d_inputs(W.scaled(W.BATCH_2D, nx=800, nz=100)), W.batch_2d_inputs(W.scaled(W.BATCH_2D, nx=800, nz=100))
    assert np.array_equal(a["v_true"], b["v_true"])
    assert [s["width"] for s in a["shots"]] == [s["width"] for s in b["shots"]]
    assert np.array_equal(W.faulted_layers(300, 200, 5), W.faulted_layers(300, 200, 5))
    assert not np.array_equal(W.faulted_layers(300, 200, 5), W.faulted_layers(300, 200, 6))
    assert np.array_equal(W.random_field((4, 5), 3), W.random_field((4, 5), 3))


def test_ricker_peak_frequency():
    # the wavelet's amplitude spectrum peaks at its peak frequency (R11)
    w = W.SMALL_2D
    r = W.ricker(4000, w.dt, w.f_peak)
    f = np.fft.rfftfreq(len(r), w.dt)
    assert f[np.argmax(np.abs(np.fft.rfft(r)))] == pytest.approx(w.f_peak, abs=0.5)
