"""Pins for the oracle's RTM with wavefield storage (Algorithm 2) with the
source wavefield kept every k steps (Eq. 7's Nyquist step).

* brute force: the dense-matrix pipeline of test_oracle_rtm (Kronecker
  Laplacian, stored forward levels) with the imaging sums restricted to the
  kept levels; the stored fields themselves against the dense forward levels;
* Eq. 7 and the storage figures the paper prints (the 5 ms Nyquist step of
  the 2-D RTM, the 132.062 GB of the 3-D storage RTM and its 300.82 ratio to
  the two reconstruction panels);
* stride 1 against Algorithm 3 (reconstruction) on a random boundary: the
  paper's premise that both RTM variants form the same image;
* with k at Eq. 7's step the sampled integrals stay close to the full ones,
  and a stride well beyond it does not.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_rtm import dense_laplacian, flat

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dense_storage(a_true, a_mig, h, nt, src, wav, rec, nb, interior, stride):
    shape = a_true.shape
    ndim = len(shape)
    Lm = dense_laplacian(shape, np.array([-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]))
    scale = h ** (2 - ndim)
    s = flat(shape, src)
    R = [flat(shape, r) for r in rec]

    def forward(a):
        A = a.ravel()
        P = [np.zeros(A.size), np.zeros(A.size)]
        for n in range(nt):
            nxt = 2 * P[-1] - P[-2] + A * (Lm @ P[-1])
            nxt[s] -= A[s] * wav[n] * scale
            P.append(nxt)
        return P[1:]

    seis = np.array([[p[r] for p in forward(a_true)] for r in R])
    P = forward(a_mig)
    A = a_mig.ravel()
    Q = {nt + 1: np.zeros(A.size), nt: np.zeros(A.size)}
    for n in range(nt, 0, -1):
        nxt = 2 * Q[n] - Q[n + 1] + A * (Lm @ Q[n])
        for k, r in enumerate(R):
            nxt[r] += A[r] * seis[k, n] * scale
        Q[n - 1] = nxt
    kept = range(0, nt + 1, stride)
    nx, ny, nz = interior
    win = ((slice(nb, nb + nz), slice(nb, nb + nx)) if ndim == 2 else
           (slice(nb, nb + nz), slice(nb, nb + ny), slice(nb, nb + nx)))
    num = sum(P[n] * Q[n] for n in kept).reshape(shape)[win]
    den = sum(P[n] * P[n] for n in kept).reshape(shape)[win]
    store = np.array([P[n].reshape(shape)[win] for n in kept])
    return seis, num, den, store


def _tiny(ndim, seed):
    rng = np.random.default_rng(seed)
    if ndim == 2:
        nx, ny, nz, nb = 8, 1, 6, 3
        shape = (nz + 2 * nb, nx + 2 * nb)
        src = np.array([nb + 4, 0, nb + 1], np.int32)
        rec = np.array([[nb + i, 0, nb + 1] for i in range(nx)], np.int32)
    else:
        nx, ny, nz, nb = 5, 4, 4, 3
        shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
        src = np.array([nb + 2, nb + 1, nb + 1], np.int32)
        rec = np.array([[nb + i, nb + j, nb + 1] for j in range(ny) for i in range(nx)], np.int32)
    return rng, (nx, ny, nz), nb, shape, src, rec


@pytest.mark.parametrize("ndim,stride", [(2, 1), (2, 3), (2, 7), (3, 4)])
def test_bruteforce_storage_rtm(ndim, stride):
    rng, interior, nb, shape, src, rec = _tiny(ndim, 20 + stride)
    a_true = rng.uniform(0.05, 0.2, shape)
    a_mig = rng.uniform(0.05, 0.2, shape)
    h, nt = 7.0, 29            # nt not a multiple of the stride: a ragged last interval
    wav = rng.standard_normal(nt)
    seis, num_d, den_d, store_d = dense_storage(a_true, a_mig, h, nt, src, wav, rec, nb, interior, stride)
    r = oracle.rtm_storage(a_mig, h, nt, src, wav, rec, seis, nb, interior, stride, keep_store=True)
    assert r["store"].shape[0] == nt // stride + 1
    np.testing.assert_allclose(r["store"], store_d, rtol=1e-10, atol=1e-12 * np.abs(store_d).max())
    np.testing.assert_allclose(r["num"], num_d, rtol=1e-10, atol=1e-11 * np.abs(num_d).max())
    np.testing.assert_allclose(r["den"], den_d, rtol=1e-10, atol=1e-11 * np.abs(den_d).max())


def test_bruteforce_catches_imaging_at_every_level():
    # summing all levels instead of the kept ones (a dropped stride test) must fail
    rng, interior, nb, shape, src, rec = _tiny(2, 3)
    a = rng.uniform(0.05, 0.2, shape)
    wav = rng.standard_normal(29)
    seis, num3, _, _ = dense_storage(a, a, 7.0, 29, src, wav, rec, nb, interior, 3)
    r1 = oracle.rtm_storage(a, 7.0, 29, src, wav, rec, seis, nb, interior, 1)
    assert np.linalg.norm(r1["num"] - num3) > 1e-2 * np.linalg.norm(num3)


def test_nyquist_step_of_eq7():
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["nyquist_step_2d"]
    assert oracle.nyquist_stride(g["dt"], g["f_max"], g["f_min"]) == g["stride"]
    assert g["stride"] * g["dt"] == pytest.approx(g["dt_nyq_printed"])
    assert oracle.nyquist_stride(0.001, 50.0, 0.0) == 10
    assert oracle.nyquist_stride(0.001, 40.0, 10.0) == 16          # band width, not f_max
    assert oracle.nyquist_stride(0.004, 1000.0) == 1               # never below one step
    assert oracle.nyquist_stride(0.001, 10.0, 20.0) == 0           # bad band


def test_storage_size_matches_section_5():
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["storage_3d"]
    nt = int(round(g["t_max"] / g["dt"]))
    k = oracle.nyquist_stride(g["dt"], 1.0 / (2 * g["dt_nyq"]))
    assert k == 10
    fields = nt // k + 1                                           # levels 0, k, ..., N
    gib = fields * int(np.prod(g["grid"])) * g["bytes_per_value"] / 2 ** 30
    assert gib == pytest.approx(g["gb_printed"], abs=5e-4)
    assert gib / g["wr_gb_printed"] == pytest.approx(g["ratio_printed"], abs=5e-3)


def test_stride_one_equals_reconstruction_rtm():
    # Algorithm 2 with every level stored and Algorithm 3 (exact reconstruction
    # through the random boundary) form the same integrals
    w = W.scaled(W.SMALL_2D, nx=60, nz=50, nb=20, nt=400, name="st1")
    v = W.three_layers(w.nx, w.nz)
    a = oracle.coef(oracle.rbc_velocity(v, w.nb, w.v_lo, w.v_hi, w.v_max, 3), w.dt, w.h)[1].astype(float)
    src, rec = W.source_at(w, w.nx // 2), W.surface_line(w)
    wav = W.ricker(w.nt, w.dt, w.f_peak)
    seis = oracle.model(a, w.h, w.nt, src, wav, rec)["seis"]
    rs = oracle.rtm_storage(a, w.h, w.nt, src, wav, rec, seis, w.nb, (w.nx, 1, w.nz), 1)
    rr = oracle.rtm_shot(a, w.h, w.nt, src, wav, rec, seis, w.nb, (w.nx, 1, w.nz))
    for key in ("num", "den"):
        assert np.linalg.norm(rs[key] - rr[key]) <= 1e-9 * np.linalg.norm(rr[key])


def test_nyquist_stride_keeps_the_image():
    # the integrals sampled at Eq. 7's step (f_max = 2.5 f_peak) stay close to
    # the full integrals; 4x that stride aliases
    w = W.scaled(W.SMALL_2D, nx=100, nz=80, nb=25, nt=700, name="nyq")
    v = W.three_layers(w.nx, w.nz)
    a = oracle.coef(oracle.rbc_velocity(v, w.nb, w.v_lo, w.v_hi, w.v_max, 3), w.dt, w.h)[1].astype(float)
    am = oracle.coef(oracle.rbc_velocity(W.smooth_slowness(v, 4.0), w.nb, w.v_lo, w.v_hi, w.v_max, 3),
                     w.dt, w.h)[1].astype(float)
    src, rec = W.source_at(w, w.nx // 2), W.surface_line(w)
    wav = W.ricker(w.nt, w.dt, w.f_peak)
    seis = oracle.model(a, w.h, w.nt, src, wav, rec)["seis"]
    k = oracle.nyquist_stride(w.dt, 2.5 * w.f_peak)
    assert k > 5
    full = oracle.rtm_storage(am, w.h, w.nt, src, wav, rec, seis, w.nb, (w.nx, 1, w.nz), 1)
    ref = oracle.image(full["num"], full["den"])

    def err(stride):
        r = oracle.rtm_storage(am, w.h, w.nt, src, wav, rec, seis, w.nb, (w.nx, 1, w.nz), stride)
        return np.linalg.norm(oracle.image(r["num"], r["den"]) - ref) / np.linalg.norm(ref)

    e_nyq, e_alias = err(k), err(4 * k)
    assert e_nyq < 1e-2
    assert e_alias > 5 * e_nyq
