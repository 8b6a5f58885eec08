"""Pins for the oracle's modeling (Algorithm 1), RTM with wavefield
reconstruction (Algorithm 3, Eqs. 2, 3, 6) and stacking.

* brute force: on tiny grids the whole pipeline is recomputed with dense
  matrices (L = sum of Kronecker products of the banded Toeplitz second
  difference), and the image is formed from STORED forward wavefields
  (Algorithm 2) instead of the reconstruction -- the paper's claim that the
  two RTM variants give the same image;
* exact reversibility (Section 4.3, Figure 1: the undamped random boundary
  keeps all energy, so p^R reproduces p);
* the image sign (Eq. 3: the image carries the sign of the reflection
  coefficient) on a flat reflector.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def toeplitz_d2(n, c):
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - 4), min(n, i + 5)):
            D[i, j] = c[abs(i - j)]
    return D


def dense_laplacian(shape, c):
    """h^2 lap as a dense matrix on a z-major flattened grid, zero outside."""
    if len(shape) == 2:
        nz, nx = shape
        return np.kron(np.eye(nz), toeplitz_d2(nx, c)) + np.kron(toeplitz_d2(nz, c), np.eye(nx))
    nz, ny, nx = shape
    I = np.eye
    return (np.kron(I(nz), np.kron(I(ny), toeplitz_d2(nx, c)))
            + np.kron(I(nz), np.kron(toeplitz_d2(ny, c), I(nx)))
            + np.kron(toeplitz_d2(nz, c), np.kron(I(ny), I(nx))))


def flat(shape, node):
    x, y, z = node
    if len(shape) == 2:
        return z * shape[1] + x
    return (z * shape[1] + y) * shape[2] + x


def dense_pipeline(a_true, a_mig, h, nt, src, wav, rec, nb, interior, rec_sign=1.0):
    shape = a_true.shape
    ndim = len(shape)
    c = np.array([-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560])
    # the weights themselves are pinned in test_oracle_stencil; here only the
    # matrix assembly differs from the oracle's loops
    Lm = dense_laplacian(shape, c)
    scale = h ** (2 - ndim)
    s = flat(shape, src)
    R = [flat(shape, r) for r in rec]

    def forward(a):
        A = a.ravel()
        P = [np.zeros(A.size), np.zeros(A.size)]   # p^{-1}, p^0
        for n in range(nt):
            nxt = 2 * P[-1] - P[-2] + A * (Lm @ P[-1])
            nxt[s] -= A[s] * wav[n] * scale
            P.append(nxt)
        return P[1:]                                # p^0 .. p^nt

    seis = np.array([[p[r] for p in forward(a_true)] for r in R])
    P = forward(a_mig)                              # stored wavefields (Algorithm 2)
    A = a_mig.ravel()
    Q = {nt + 1: np.zeros(A.size), nt: np.zeros(A.size)}
    for n in range(nt, 0, -1):
        nxt = 2 * Q[n] - Q[n + 1] + A * (Lm @ Q[n])
        for k, r in enumerate(R):
            nxt[r] += rec_sign * A[r] * seis[k, n] * scale
        Q[n - 1] = nxt
    nx, ny, nz = interior
    num = sum(P[n] * Q[n] for n in range(nt + 1)).reshape(shape)
    den = sum(P[n] * P[n] for n in range(nt + 1)).reshape(shape)
    if ndim == 2:
        win = (slice(nb, nb + nz), slice(nb, nb + nx))
    else:
        win = (slice(nb, nb + nz), slice(nb, nb + ny), slice(nb, nb + nx))
    return seis, num[win], den[win]


@pytest.mark.parametrize("ndim", [2, 3])
def test_bruteforce_modeling_and_rtm(ndim):
    rng = np.random.default_rng(10 + ndim)
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
    a_true = rng.uniform(0.05, 0.2, shape)
    a_mig = rng.uniform(0.05, 0.2, shape)
    h, nt = 7.0, 30
    wav = rng.standard_normal(nt)
    seis_d, num_d, den_d = dense_pipeline(a_true, a_mig, h, nt, src, wav, rec, nb, (nx, ny, nz))
    seis = oracle.model(a_true, h, nt, src, wav, rec)["seis"]
    np.testing.assert_allclose(seis, seis_d, rtol=1e-12, atol=1e-12 * np.abs(seis_d).max())
    r = oracle.rtm_shot(a_mig, h, nt, src, wav, rec, seis, nb, (nx, ny, nz))
    np.testing.assert_allclose(r["num"], num_d, rtol=1e-10, atol=1e-11 * np.abs(num_d).max())
    np.testing.assert_allclose(r["den"], den_d, rtol=1e-10, atol=1e-11 * np.abs(den_d).max())


def test_bruteforce_catches_a_one_step_time_shift():
    # pairing p^R_n with pbar_{n-1} (an off-by-one in the reverse loop) must fail
    rng = np.random.default_rng(5)
    nx, nz, nb = 8, 6, 3
    shape = (nz + 2 * nb, nx + 2 * nb)
    src = np.array([nb + 4, 0, nb + 1], np.int32)
    rec = np.array([[nb + i, 0, nb + 1] for i in range(nx)], np.int32)
    a = rng.uniform(0.05, 0.2, shape)
    wav = rng.standard_normal(30)
    seis = oracle.model(a, 7.0, 30, src, wav, rec)["seis"]
    shifted = np.concatenate([seis[:, 1:], np.zeros((nx, 1))], 1)   # planted mistake
    _, num_d, _ = dense_pipeline(a, a, 7.0, 30, src, wav, rec, nb, (nx, 1, nz))
    r = oracle.rtm_shot(a, 7.0, 30, src, wav, rec, shifted, nb, (nx, 1, nz))
    assert np.linalg.norm(r["num"] - num_d) > 1e-3 * np.linalg.norm(num_d)


def _rbc_case(ndim, seed=1):
    if ndim == 2:
        w = W.scaled(W.SMALL_2D, nx=80, nz=60, nb=20, nt=500, name="rev2")
        v = np.full((w.nz, w.nx), 2000.0)
    else:
        w = W.scaled(W.SHOT_3D, nx=24, ny=22, nz=20, nb=10, nt=150, name="rev3")
        v = np.full((w.nz, w.ny, w.nx), 2000.0)
    vp = oracle.rbc_velocity(v, w.nb, w.v_lo, w.v_hi, w.v_max, seed)
    a = oracle.coef(vp, w.dt, w.h)[1].astype(np.float64)
    src = W.source_at(w, w.nx // 2, w.ny // 2 if ndim == 3 else 0, depth=w.nz // 3)
    return w, a, src


@pytest.mark.parametrize("ndim", [2, 3])
def test_exact_time_reversibility_with_random_boundary(ndim):
    w, a, src = _rbc_case(ndim)
    wav = W.ricker(w.nt, w.dt, w.f_peak)
    snaps = [0, 10, w.nt // 4, w.nt // 2, w.nt - 1, w.nt]
    fwd = oracle.model(a, w.h, w.nt, src, wav, np.zeros((0, 3), np.int32), snaps=snaps)["snaps"]
    interior = (w.nx, w.ny if ndim == 3 else 1, w.nz)
    r = oracle.rtm_shot(a, w.h, w.nt, src, wav, np.zeros((0, 3), np.int32),
                        np.zeros((0, w.nt + 1)), w.nb, interior, snaps=snaps)
    ref = np.linalg.norm(fwd[3])
    for k, n in enumerate(snaps):
        assert np.linalg.norm(r["pr"][k] - fwd[k]) <= 1e-10 * ref, n


def test_literal_eq6_reconstructs_only_after_the_source_stops():
    # without re-subtracting the source, p^R matches p once the wavelet is over,
    # and not while it is still active
    w, a, src = _rbc_case(2)
    wav = W.ricker(w.nt, w.dt, w.f_peak)   # 15 Hz: support ends near 0.2 s = step 200
    snaps = [50, 300, w.nt]
    fwd = oracle.model(a, w.h, w.nt, src, wav, np.zeros((0, 3), np.int32), snaps=snaps)["snaps"]
    r = oracle.rtm_shot(a, w.h, w.nt, src, wav, np.zeros((0, 3), np.int32),
                        np.zeros((0, w.nt + 1)), w.nb, (w.nx, 1, w.nz), reinject=False,
                        snaps=snaps)
    ref = np.linalg.norm(fwd[1])
    assert np.linalg.norm(r["pr"][2] - fwd[2]) <= 1e-10 * ref
    assert np.linalg.norm(r["pr"][1] - fwd[1]) <= 1e-6 * ref
    assert np.linalg.norm(r["pr"][0] - fwd[0]) > 1e-2 * np.linalg.norm(fwd[0])


def test_flat_reflector_image_has_the_sign_of_the_reflection_coefficient():
    # v: 2000 over 3000 m/s at interior depth 60 -> R = (3000-2000)/(3000+2000) > 0;
    # migrate the reflected data (total minus direct) in the upper velocity
    w = W.scaled(W.SMALL_2D, nx=120, nz=120, nb=30, nt=700, name="refl")
    v = W.two_layers(w.nx, w.nz, 60, 2000.0, 3000.0)
    vm = np.full_like(v, 2000.0)
    a = oracle.coef(oracle.rbc_velocity(v, w.nb, 1500, 3000, 3000, 1), w.dt, w.h)[1].astype(float)
    am = oracle.coef(oracle.rbc_velocity(vm, w.nb, 1500, 3000, 3000, 1), w.dt, w.h)[1].astype(float)
    src, rec = W.source_at(w, w.nx // 2), W.surface_line(w)
    wav = W.ricker(w.nt, w.dt, w.f_peak)
    d = oracle.model(a, w.h, w.nt, src, wav, rec)["seis"] - oracle.model(am, w.h, w.nt, src, wav, rec)["seis"]
    r = oracle.rtm_shot(am, w.h, w.nt, src, wav, rec, d, w.nb, (w.nx, 1, w.nz))
    img = oracle.image(r["num"], r["den"])
    prof = img[:, w.nx // 2 - 20: w.nx // 2 + 20].mean(1)
    half_wl = int(np.ceil(2000.0 / w.f_peak / w.h / 2))      # ~7 cells
    peak = np.argmax(np.abs(prof[10:])) + 10
    assert abs(peak - 60) <= half_wl
    assert prof[peak] > 0


def test_image_ratio_and_stack_properties():
    rng = np.random.default_rng(2)
    p, pb = rng.standard_normal((5, 7)), rng.standard_normal((5, 7))
    # one time sample: Eq. 3 reduces to pbar / p
    np.testing.assert_allclose(oracle.image(p * pb, p * p, 0.0), pb / p, rtol=1e-14)
    # the ratio is unchanged by a common scale of num and den
    num, den = rng.standard_normal((4, 6)), rng.uniform(0.5, 2, (4, 6))
    np.testing.assert_allclose(oracle.image(3 * num, 3 * den), oracle.image(num, den), rtol=1e-13)
    # eps damps where den is small relative to its maximum
    img = oracle.image(np.ones(3), np.array([1.0, 1e-9, 0.0]), 1e-6)
    assert img[0] == pytest.approx(1 / (1 + 1e-6)) and img[2] == pytest.approx(1e6)
    survey = np.zeros((4, 20))
    oracle.stack(survey, np.ones((4, 6)), 3)
    oracle.stack(survey, 2 * np.ones((4, 6)), 6)
    ref = np.zeros((4, 20)); ref[:, 3:9] += 1; ref[:, 6:12] += 2
    np.testing.assert_array_equal(survey, ref)
