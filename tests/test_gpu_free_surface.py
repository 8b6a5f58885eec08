"""The free-surface option (Section 5: a pressure-release top of 4 zero rows,
the random boundary on the sides and the bottom) on the GPU through the C ABI
against the FP64 oracle: the padded coefficient, modeling, both RTM
algorithms, 2-D and 3-D.  Tolerance: relative L2 <= 1e-4."""
import numpy as np
import pytest

import oracle
import workloads as W
from rtm_cases import TOL, f32, rel, rel_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import paper_2204_03380_gb300 as R
    return R


def fs_case(ndim, nx, ny, nz, nb, nt, seed=0):
    base = W.SMALL_2D if ndim == 2 else W.SHOT_3D
    w = W.scaled(base, nx=nx, ny=ny, nz=nz, nb=nb, nt=nt, name="fs")
    w = W.dataclasses.replace(w, rbc_seed=seed + 11)
    v = (W.three_layers(nx, nz, (nz // 3, 2 * nz // 3)) if ndim == 2 else W.dipping_salt_3d(nx, ny, nz, seed + 2))
    cy = (nb + ny // 2) if ndim == 3 else 0
    src = np.array([nb + nx // 2, cy, 4 + 1], np.int32)           # just below the surface rows
    if ndim == 2:
        rec = np.array([[nb + i, 0, 4] for i in range(0, nx, 2)], np.int32)
    else:
        rec = np.array([[nb + i, nb + j, 4] for j in range(0, ny, 3) for i in range(0, nx, 3)], np.int32)
    return w, v, src, rec, W.ricker(nt, w.dt, w.f_peak)


def grid(R, w):
    return R.make_grid(w.ndim, w.nx, w.ny, w.nz, w.nb, w.h, w.dt, w.nt, free_surface=1)


def gpu_a(R, w, v):
    g = grid(R, w)
    a = torch.empty(g.padded, dtype=torch.float32, device="cuda")
    vp = torch.empty(g.padded, dtype=torch.float32, device="cuda")
    R.rbc_build_velocity(g, torch.tensor(np.asarray(v, np.float32), device="cuda"), w.v_lo, w.v_hi, w.v_max,
                         w.rbc_seed, 0, vp, a)
    return g, a, vp


def oracle_a(w, v):
    vp = oracle.rbc_velocity(f32(v), w.nb, w.v_lo, w.v_hi, w.v_max, w.rbc_seed, free_surface=True)
    return vp, oracle.coef(vp, w.dt, w.h)[1]


def run(R, w, v, src, rec, wav, stride=None):
    g, a, vp = gpu_a(R, w, v)
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    seis = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
    num = torch.zeros(g.interior, dtype=torch.float32, device="cuda")
    den = torch.zeros_like(num)
    ctx = R.rbc_create(g, a)
    try:
        R.rbc_model(ctx, src, wt, rec, seis)
        if stride is None:
            R.rbc_rtm_shot(ctx, src, wt, rec, seis, R.RBC_REINJECT_SOURCE, num, den)
        else:
            store = torch.empty(R.rbc_storage_bytes(g, stride) // 4, dtype=torch.float32, device="cuda")
            R.rbc_rtm_storage(ctx, src, wt, rec, seis, stride, store, 0, num, den)
        img = torch.zeros_like(num)
        R.rbc_image_stack(g, num, den, 1e-6, 0, 0, g, img)
        torch.cuda.synchronize()
    finally:
        R.rbc_destroy(ctx)
    return dict(a=a.cpu().numpy(), vp=vp.cpu().numpy(), seis=seis.cpu().numpy(), num=num.cpu().numpy(),
                den=den.cpu().numpy(), img=img.cpu().numpy())


def run_oracle(w, v, src, rec, wav, seis, stride=None):
    vp, a32 = oracle_a(w, v)
    a = a32.astype(np.float64)
    m = oracle.model(a, w.h, w.nt, src, f32(wav), rec)
    interior = (w.nx, w.ny if w.ndim == 3 else 1, w.nz)
    if stride is None:
        r = oracle.rtm_shot(a, w.h, w.nt, src, f32(wav), rec, f32(seis), w.nb, interior, top=4)
    else:
        r = oracle.rtm_storage(a, w.h, w.nt, src, f32(wav), rec, f32(seis), w.nb, interior, stride, top=4)
    return dict(vp=vp, a=a32, seis=m["seis"], num=r["num"], den=r["den"], img=oracle.image(r["num"], r["den"]))


@pytest.mark.parametrize("dims,stride", [((2, 150, 1, 90, 20, 700), None), ((2, 150, 1, 90, 20, 700), 5),
                                         ((3, 30, 26, 24, 6, 200), None)])
def test_free_surface_matches_oracle(R, dims, stride):
    w, v, src, rec, wav = fs_case(*dims)
    g = run(R, w, v, src, rec, wav, stride)
    o = run_oracle(w, v, src, rec, wav, g["seis"], stride)
    assert g["a"].shape == o["a"].shape == grid(R, w).padded
    np.testing.assert_allclose(g["a"], o["a"], rtol=1.2e-7, atol=0)
    assert np.all(g["a"][:4] == 0) and np.all(g["vp"][:4] == 0)
    assert rel(g["seis"], o["seis"]) <= TOL
    assert rel(g["num"], o["num"]) <= TOL
    assert rel(g["den"], o["den"]) <= TOL
    e, frac = rel_image(g["img"], o["img"], o["den"])
    assert e <= TOL and frac > 0.05, (e, frac)


def test_free_surface_is_not_offered_where_not_built(R):
    w, v, src, rec, wav = fs_case(2, 40, 1, 30, 6, 50)
    g, a, _ = gpu_a(R, w, v)
    ctx = R.rbc_create(g, a)
    try:
        d = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
        with pytest.raises(R.RBCError, match="ENOTSUP"):
            R.rbc_fwi_forward(ctx, src, torch.tensor(np.asarray(wav, np.float32), device="cuda"), rec, d,
                              torch.zeros_like(d), torch.zeros(1, dtype=torch.float64, device="cuda"))
    finally:
        R.rbc_destroy(ctx)
    with pytest.raises((R.RBCError, ValueError)):
        R.rbc_batch_create(g, [w.nx], [a])
