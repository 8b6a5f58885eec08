"""RTM with wavefield storage (Algorithm 2, Eq. 7 stride) on the GPU through
the C ABI against the FP64 oracle: the stored levels, the two sampled
integrals of Eq. 3 and the image.  Tolerance: relative L2 <= 1e-4."""
import numpy as np
import pytest

import oracle
import workloads as W
from rtm_cases import TOL, case_2d, case_3d, f32, gpu_build, oracle_a, rel, rel_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import paper_2204_03380_gb300 as R
    return R


def run_gpu(R, w, v, src, rec, wav, strides, v_rtm=None):
    """Model with v, then migrate with v_rtm by Algorithm 2 for each stride in
    turn on one context (each new stride re-captures the storage graphs)."""
    g, a, _ = gpu_build(R, torch, w, v)
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    rec = np.asarray(rec, np.int32).reshape(-1, 3)
    seis = torch.zeros((rec.shape[0], w.nt + 1), dtype=torch.float32, device="cuda")
    ctx = R.rbc_create(g, a)
    try:
        R.rbc_model(ctx, src, wt, rec, seis)
    finally:
        R.rbc_destroy(ctx)
    if v_rtm is not None:
        g, a, _ = gpu_build(R, torch, w, v_rtm)
    out = []
    ctx = R.rbc_create(g, a)
    try:
        for k in strides:
            nbytes = R.rbc_storage_bytes(g, k)
            store = torch.full((nbytes // 4,), float("nan"), dtype=torch.float32, device="cuda")
            num = torch.zeros(g.interior, dtype=torch.float32, device="cuda")
            den = torch.zeros_like(num)
            R.rbc_rtm_storage(ctx, src, wt, rec, seis, k, store, 0, num, den)
            img = torch.zeros_like(num)
            R.rbc_image_stack(g, num, den, 1e-6, 0, 0, g, img)
            torch.cuda.synchronize()
            out.append(dict(store=store.view((w.nt // k + 1,) + g.interior).cpu().numpy(),
                            num=num.cpu().numpy(), den=den.cpu().numpy(), img=img.cpu().numpy()))
    finally:
        R.rbc_destroy(ctx)
    return out, seis.cpu().numpy()


def run_oracle(w, v_rtm, src, rec, wav, seis, k):
    a = oracle_a(w, v_rtm)[1].astype(np.float64)
    r = oracle.rtm_storage(a, w.h, w.nt, src, f32(wav), rec, f32(seis), w.nb,
                           (w.nx, w.ny if w.ndim == 3 else 1, w.nz), k, keep_store=True)
    r["img"] = oracle.image(r["num"], r["den"], 1e-6)
    return r


def check(g, o):
    scale = max(np.linalg.norm(x) for x in o["store"])
    assert max(np.linalg.norm(a - b) for a, b in zip(g["store"], o["store"])) <= TOL * scale
    assert rel(g["num"], o["num"]) <= TOL
    assert rel(g["den"], o["den"]) <= TOL
    e, frac = rel_image(g["img"], o["img"], o["den"])
    assert e <= TOL and frac > 0.05, (e, frac)


@pytest.mark.parametrize("case", [("config1_full", 200, 200, 50, 1000), ("ragged", 37, 23, 6, 401)],
                         ids=lambda c: c[0])
def test_2d_storage_rtm_matches_oracle(R, case):
    w, v, src, rec, wav = case_2d(*case)
    vm = W.smooth_slowness(v, 4.0)
    k_nyq = R.rbc_nyquist_stride(w.dt, 2.5 * w.f_peak)
    strides = (1, k_nyq, 7)
    g, seis = run_gpu(R, w, v, src, rec, wav, strides, v_rtm=vm)
    for gk, k in zip(g, strides):
        check(gk, run_oracle(w, vm, src, rec, wav, seis, k))


def test_3d_storage_rtm_matches_oracle(R):
    w, v, src, rec, wav = case_3d("st3", 30, 26, 40, 6, 203)
    g, seis = run_gpu(R, w, v, src, rec, wav, (4,))
    check(g[0], run_oracle(w, v, src, rec, wav, seis, 4))


def test_stride_one_matches_reconstruction_rtm_on_gpu(R):
    # Algorithm 2 with every level stored and Algorithm 3 (reconstruction)
    w, v, src, rec, wav = case_2d("st1", 120, 90, 20, 600)
    g, seis = run_gpu(R, w, v, src, rec, wav, (1,))
    gg, a, _ = gpu_build(R, torch, w, v)
    ctx = R.rbc_create(gg, a)
    try:
        num = torch.zeros(gg.interior, dtype=torch.float32, device="cuda")
        den = torch.zeros_like(num)
        wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
        R.rbc_rtm_shot(ctx, src, wt, rec, torch.tensor(seis, device="cuda"), R.RBC_REINJECT_SOURCE, num, den)
        torch.cuda.synchronize()
    finally:
        R.rbc_destroy(ctx)
    assert rel(g[0]["num"], num.cpu().numpy()) <= TOL
    assert rel(g[0]["den"], den.cpu().numpy()) <= TOL


def test_storage_argument_errors(R):
    w, v, src, rec, wav = case_2d("err", 30, 20, 4, 50)
    g, a, _ = gpu_build(R, torch, w, v)
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    seis = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
    num = torch.zeros(g.interior, dtype=torch.float32, device="cuda")
    den = torch.zeros_like(num)
    ctx = R.rbc_create(g, a)
    try:
        small = torch.zeros(R.rbc_storage_bytes(g, 5) // 4 - 1, dtype=torch.float32, device="cuda")
        with pytest.raises(R.RBCError, match="EINVAL"):
            R.rbc_rtm_storage(ctx, src, wt, rec, seis, 5, small, 0, num, den)
        with pytest.raises(R.RBCError, match="EINVAL"):
            R.rbc_rtm_storage(ctx, src, wt, rec, seis, 0, small, 0, num, den)
        ok = torch.zeros(R.rbc_storage_bytes(g, 5) // 4, dtype=torch.float32, device="cuda")
        with pytest.raises(R.RBCError, match="EINVAL"):
            R.rbc_rtm_storage(ctx, src, wt, rec, seis, 5, ok, R.RBC_REINJECT_SOURCE, num, den)
        R.rbc_rtm_storage(ctx, src, wt, rec, seis, 5, ok, R.RBC_ZERO_FIRST, num, den)
        torch.cuda.synchronize()
        assert np.all(num.cpu().numpy() == 0)   # no receivers' data: pbar stays 0
    finally:
        R.rbc_destroy(ctx)
