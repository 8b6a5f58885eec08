"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds input data only -- interior velocity models, the source
wavelet, shot/receiver geometry and the workload presets -- and none of the
method's arithmetic (no stencil, no random boundary, no imaging).  The paper's
own benchmarks (2-D Marmousi, HPC4E MODEL AF; Section 5) are not available, so
these seeded models stand in for them with the same kinds of structure: flat,
dipping and faulted layers, a high-velocity salt-like body, a smoothed
migration model, a Ricker source near the surface and a fixed-spread surface
receiver line or grid.

Coordinates: padded grid nodes (x, y, z), z down, x fastest in memory; the
interior starts at node nb on every axis.  2-D arrays are (nz, nx) and 3-D
arrays (nz, ny, nx).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


# --------------------------------------------------------------------------
# workload presets
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    ndim: int
    nx: int
    ny: int
    nz: int
    nb: int
    h: float
    dt: float
    nt: int
    f_peak: float
    v_lo: float          # random-boundary velocity range
    v_hi: float
    v_max: float         # cap (model maximum; keeps the scheme stable)
    rbc_seed: int
    nshots: int = 1

    @property
    def padded(self):
        n = 2 * self.nb
        if self.ndim == 2:
            return (self.nz + n, self.nx + n)
        return (self.nz + n, self.ny + n, self.nx + n)

    @property
    def npad(self) -> int:
        return int(np.prod(self.padded))


# one 2-D shot on three flat layers, 200 x 200 interior + 50-cell boundary
SMALL_2D = Workload("2d_200x200_nb50_1000steps", 2, 200, 1, 200, 50, 10.0, 1e-3, 1000,
                    15.0, 1500.0, 4500.0, 3500.0, 1)
# 240-shot 2-D survey on a faulted layered model, 2301 x 751 + 60-cell boundary
SURVEY_2D = Workload("2d_2301x751_nb60_12500steps_240shots", 2, 2301, 1, 751, 60, 4.0,
                     0.4e-3, 12500, 25.0, 1500.0, 5500.0, 5500.0, 2, nshots=240)
# one 3-D shot, 500 x 500 x 300 + 40-cell boundary
SHOT_3D = Workload("3d_500x500x300_nb40_3000steps", 3, 500, 500, 300, 40, 10.0, 1e-3, 3000,
                   15.0, 1500.0, 4500.0, 4500.0, 3)


# 64 shots of uneven aperture (400-1200 columns) over a 4000 x 600 model at 5 m
BATCH_2D = Workload("2d_batch_64shots_w400-1200_600rows_nb50_3000steps", 2, 4000, 1, 600, 50, 5.0,
                    0.5e-3, 3000, 25.0, 1500.0, 4000.0, 4000.0, 4, nshots=64)

# FWI gradient: 300 x 300 three-layer model with a Gaussian velocity anomaly,
# 10 m cells, 50-cell random boundary, 1000 steps of 1 ms, 15 Hz, 4 shots
FWI_2D = Workload("2d_fwi_300x300_nb50_1000steps_4shots", 2, 300, 1, 300, 50, 10.0, 1e-3, 1000,
                  15.0, 1500.0, 4500.0, 3500.0, 1, nshots=4)


def scaled(w: Workload, nx=None, ny=None, nz=None, nb=None, nt=None, name=None) -> Workload:
    """A smaller copy of a preset (same spacing, velocities and source)."""
    return dataclasses.replace(
        w, nx=nx or w.nx, ny=ny or w.ny, nz=nz or w.nz, nb=nb or w.nb, nt=nt or w.nt,
        name=name or (w.name + "_scaled"))


# --------------------------------------------------------------------------
# wavelet
# --------------------------------------------------------------------------
def ricker(nt: int, dt: float, f_peak: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet with peak frequency f_peak, delayed by t0 (default 1.5/f_peak).

    w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),  tau = t - t0,  t = n dt.
    """
    if t0 is None:
        t0 = 1.5 / f_peak
    t = np.arange(nt) * dt - t0
    x = (math.pi * f_peak * t) ** 2
    return ((1.0 - 2.0 * x) * np.exp(-x)).astype(np.float64)


# --------------------------------------------------------------------------
# interior velocity models
# --------------------------------------------------------------------------
def three_layers(nx: int, nz: int, depths=(70, 140), vels=(1500.0, 2500.0, 3500.0)) -> np.ndarray:
    """Flat layers: vels[0] above depths[0], vels[1] to depths[1], vels[2] below."""
    v = np.full((nz, nx), vels[0], np.float64)
    v[depths[0]:depths[1]] = vels[1]
    v[depths[1]:] = vels[2]
    return v


def two_layers(nx: int, nz: int, depth: int, v1: float, v2: float) -> np.ndarray:
    v = np.full((nz, nx), v1, np.float64)
    v[depth:] = v2
    return v


def faulted_layers(nx: int, nz: int, seed: int, v_min=1500.0, v_max=5500.0,
                   nlayers=12, nfaults=3) -> np.ndarray:
    """Seeded layered model with gentle dips and normal faults (2-D).

    Interfaces are random-depth lines with small random dips; each fault is a
    dipping line across which the deeper interfaces are thrown down by a random
    offset.  Velocity increases with layer index from v_min to v_max.
    """
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, :].astype(np.float64)
    z = np.arange(nz)[:, None].astype(np.float64)
    base = np.sort(rng.uniform(0.06, 0.95, nlayers - 1)) * nz
    dips = rng.uniform(-0.08, 0.08, nlayers - 1)
    shift = np.zeros((1, nx))
    faults = []
    for _ in range(nfaults):
        x0 = rng.uniform(0.15, 0.85) * nx
        slope = rng.uniform(0.4, 0.9) * rng.choice([-1, 1])
        throw = rng.uniform(0.02, 0.05) * nz
        faults.append((x0, slope, throw))
    layer = np.zeros((nz, nx), np.int32)
    for k in range(nlayers - 1):
        depth = base[k] + dips[k] * (x - nx / 2) + shift
        for (x0, slope, throw) in faults:
            # hanging wall: points right of the fault plane (x > x0 + slope*z)
            hw = x > (x0 + slope * (depth))
            depth = depth + throw * hw
        layer += (z >= depth).astype(np.int32)
    vel = np.linspace(v_min, v_max, nlayers)
    return vel[layer].astype(np.float64)


def smooth_slowness(v: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Migration model: Gaussian smoothing of the slowness 1/v (separable)."""
    from scipy.ndimage import gaussian_filter
    s = gaussian_filter(1.0 / v, sigma_cells, mode="nearest")
    return 1.0 / s


def dipping_salt_3d(nx: int, ny: int, nz: int, seed: int, v_min=1500.0, v_max=4500.0,
                    nlayers=8) -> np.ndarray:
    """Seeded 3-D model: dipping layers plus a salt-like ellipsoid at v_max."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    base = np.sort(rng.uniform(0.08, 0.92, nlayers - 1)) * nz
    dx = rng.uniform(-0.06, 0.06, nlayers - 1)
    dy = rng.uniform(-0.06, 0.06, nlayers - 1)
    layer = np.zeros((nz, ny, nx), np.int8)
    for k in range(nlayers - 1):
        depth = base[k] + dx[k] * (x - nx / 2) + dy[k] * (y - ny / 2)
        layer += (z >= depth).astype(np.int8)
    vel = np.linspace(v_min, v_max, nlayers)
    v = vel[layer]
    cx, cy, cz = nx * rng.uniform(0.4, 0.6), ny * rng.uniform(0.4, 0.6), nz * 0.55
    rx, ry, rz = nx * 0.18, ny * 0.14, nz * 0.15
    salt = ((x - cx) / rx) ** 2 + ((y - cy) / ry) ** 2 + ((z - cz) / rz) ** 2 <= 1.0
    v = np.where(salt, v_max, v)
    return v.astype(np.float64)


# --------------------------------------------------------------------------
# geometry (padded-frame nodes)
# --------------------------------------------------------------------------
# `top` is the first interior row of the padded frame: nb (random boundary on
# every side, the default) or 4 (free-surface grids).
def surface_line(w: Workload, depth: int = 1, step: int = 1, x_from: int = 0,
                 x_to: int | None = None, top: int | None = None) -> np.ndarray:
    """Receivers every `step` interior columns at interior depth `depth` (2-D)."""
    x_to = w.nx if x_to is None else x_to
    top = w.nb if top is None else top
    xs = np.arange(x_from, x_to, step) + w.nb
    return np.stack([xs, np.zeros_like(xs), np.full_like(xs, top + depth)], 1).astype(np.int32)


def surface_grid(w: Workload, depth: int = 1, step: int = 2, top: int | None = None) -> np.ndarray:
    """Receivers on a square surface grid every `step` nodes (3-D)."""
    top = w.nb if top is None else top
    xs = np.arange(0, w.nx, step) + w.nb
    ys = np.arange(0, w.ny, step) + w.nb
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    Z = np.full_like(X, top + depth)
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.int32)


def receiver_grid_m(w: Workload, start_m: float, spacing_m: float, count: int, depth: int = 1,
                    top: int | None = None) -> np.ndarray:
    """Receivers at r = start + spacing (i - 1), i = 1..count, metres from the
    model origin on both surface axes (the form of the paper's 3-D acquisition,
    Eqs. 8-9), each at the nearest interior node (a position half-way between
    nodes goes to the next node); nodes outside the model are dropped (3-D)."""
    top = w.nb if top is None else top
    r = start_m + spacing_m * np.arange(count)
    idx = np.floor(r / w.h + 0.5).astype(np.int64)  # nearest node, halves up (the paper's sit on half nodes)
    ix = idx[(idx >= 0) & (idx < w.nx)]
    iy = idx[(idx >= 0) & (idx < w.ny)]
    X, Y = np.meshgrid(ix + w.nb, iy + w.nb, indexing="xy")
    Z = np.full_like(X, top + depth)
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.int32)


def source_at(w: Workload, ix: int, iy: int = 0, depth: int = 1, top: int | None = None) -> np.ndarray:
    """Source node at interior (ix, iy, depth) in the padded frame."""
    top = w.nb if top is None else top
    return np.array([ix + w.nb, (iy + w.nb) if w.ndim == 3 else 0, depth + top], np.int32)


def shot_columns(w: Workload, nshots: int) -> np.ndarray:
    """Interior x of `nshots` shots spread evenly across the model."""
    return np.floor((np.arange(nshots) + 0.5) * w.nx / nshots).astype(np.int32)


# --------------------------------------------------------------------------
# presets -> arrays
# --------------------------------------------------------------------------
def small_2d_inputs(w: Workload = SMALL_2D):
    """Three flat layers (1500/2500/3500 m/s), source at the top centre, all-x receivers."""
    d1 = int(round(w.nz * 0.35))
    d2 = int(round(w.nz * 0.70))
    v = three_layers(w.nx, w.nz, (d1, d2))
    return dict(v=v, src=source_at(w, w.nx // 2), rec=surface_line(w),
                wavelet=ricker(w.nt, w.dt, w.f_peak))


def survey_2d_inputs(w: Workload = SURVEY_2D, model_seed: int = 7):
    """Faulted layered true model, its smoothed migration model, shot list, receivers."""
    v_true = faulted_layers(w.nx, w.nz, model_seed, 1500.0, 5500.0)
    v_mig = smooth_slowness(v_true, 20.0)
    return dict(v_true=v_true, v_mig=v_mig, shots=shot_columns(w, w.nshots),
                rec=surface_line(w, step=5, x_to=5 * 460), wavelet=ricker(w.nt, w.dt, w.f_peak))


def shot_3d_inputs(w: Workload = SHOT_3D, model_seed: int = 11):
    v = dipping_salt_3d(w.nx, w.ny, w.nz, model_seed, 1500.0, 4500.0)
    return dict(v=v, src=source_at(w, w.nx // 2, w.ny // 2), rec=surface_grid(w, step=2),
                wavelet=ricker(w.nt, w.dt, w.f_peak))


def random_field(shape, seed: int, lo=-1.0, hi=1.0) -> np.ndarray:
    """Seeded uniform test field (for stencil-level parity cases)."""
    return np.random.default_rng(seed).uniform(lo, hi, shape)


def batch_2d_inputs(w: Workload = BATCH_2D, model_seed: int = 9, width_seed: int = 4,
                    wmin: int = 400, wmax: int = 1200, rec_step: int = 2):
    """Uneven-aperture shots over one faulted layered model.

    Shot s has an interior window of width U{wmin..wmax} (seeded) centred as
    close as it fits to (s + 0.5) w.nx / nshots; its source is at the window
    centre at depth 1 and its receivers every `rec_step` columns at depth 1.
    Nodes are in the shot's own padded grid."""
    v_true = faulted_layers(w.nx, w.nz, model_seed, w.v_lo, w.v_max, nlayers=10, nfaults=3)
    v_mig = smooth_slowness(v_true, 10.0)
    rng = np.random.default_rng(width_seed)
    widths = rng.integers(wmin, wmax + 1, w.nshots)
    shots = []
    for s, width in enumerate(widths):
        width = int(min(width, w.nx))
        centre = (s + 0.5) * w.nx / w.nshots
        off = int(min(max(round(centre - width / 2), 0), w.nx - width))
        xs = np.arange(0, width, rec_step) + w.nb
        rec = np.stack([xs, np.zeros_like(xs), np.full_like(xs, w.nb + 1)], 1).astype(np.int32)
        src = np.array([width // 2 + w.nb, 0, w.nb + 1], np.int32)
        shots.append(dict(width=width, off_x=off, src=src, rec=rec))
    return dict(v_true=v_true, v_mig=v_mig, shots=shots, wavelet=ricker(w.nt, w.dt, w.f_peak))


def fwi_2d_inputs(w: Workload = FWI_2D, rec_step: int = 2):
    """True model: three flat layers (boundaries at 35 % and 70 % of the
    depth) times 1 + 0.1 exp(-r^2 / (2 (nz/20)^2)) around the centre; starting
    model: its slowness smoothed over nz/20 cells; w.nshots evenly spaced
    sources at depth 1, receivers every rec_step columns at depth 1."""
    nx, nz = w.nx, w.nz
    vt = three_layers(nx, nz, (nz * 7 // 20, nz * 14 // 20))
    zz, xx = np.mgrid[0:nz, 0:nx]
    vt = vt * (1 + 0.1 * np.exp(-((zz - nz / 2) ** 2 + (xx - nx / 2) ** 2) / (2 * (nz / 20) ** 2)))
    v0 = smooth_slowness(vt, nz / 20)
    return dict(v_true=vt.astype(np.float32), v0=v0.astype(np.float32),
                srcs=[source_at(w, int(x)) for x in shot_columns(w, w.nshots)],
                rec=surface_line(w, step=rec_step),
                wavelet=ricker(w.nt, w.dt, w.f_peak).astype(np.float32))
