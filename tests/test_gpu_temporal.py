"""Temporal blocking of the 2-D forward phase (two levels per launch,
RBC_TEMPORAL=2): modeling and RTM through it give exactly the records, panels
and integrals of the single-level path (the same fp32 operations on the same
operands) and match the FP64 oracle; the FWI gradient through it matches the
single-level one (its shots' sums are accumulated by atomic adds).
Ragged grids, odd and even record lengths (an odd one ends with a
single-level step), a source at a tile corner (inside the neighbouring
tiles' aprons) and receivers on tile edges."""
import numpy as np
import pytest

import oracle
import workloads as W
from rtm_cases import TOL, case_2d, gpu_build, oracle_shot, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(R, monkeypatch, temporal, w, v, src, rec, wav):
    if temporal:
        monkeypatch.setenv("RBC_TEMPORAL", "2")
    else:
        monkeypatch.delenv("RBC_TEMPORAL", raising=False)
    g, a, _ = gpu_build(R, torch, w, v)
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    seis = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
    ctx = R.rbc_create(g, a)
    try:
        R.rbc_model(ctx, src, wt, rec, seis)
        prev = torch.zeros(g.padded, dtype=torch.float32, device="cuda")
        last = torch.zeros_like(prev)
        R.rbc_get_panels(ctx, prev, last)
        num = torch.zeros(g.interior, dtype=torch.float32, device="cuda")
        den = torch.zeros_like(num)
        for _ in range(2):   # the second call replays the captured graphs
            R.rbc_rtm_shot(ctx, src, wt, rec, seis, R.RBC_REINJECT_SOURCE | R.RBC_ZERO_FIRST, num, den)
        torch.cuda.synchronize()
    finally:
        R.rbc_destroy(ctx)
    return dict(seis=seis.cpu().numpy(), prev=prev.cpu().numpy(), last=last.cpu().numpy(),
                num=num.cpu().numpy(), den=den.cpu().numpy())


@pytest.mark.parametrize("nx,nz,nb,nt", [(150, 90, 20, 401), (200, 117, 20, 400), (37, 9, 4, 3)],
                         ids=["odd_nt", "even_nt", "tiny"])
def test_two_levels_per_launch_equal_single_level_and_oracle(nx, nz, nb, nt, monkeypatch):
    import paper_2204_03380_gb300 as R
    w, v, _, _, _ = case_2d("temporal", nx, nz, nb, nt, seed=3, layered=False)
    wav = W.ricker(nt + 90, w.dt, w.f_peak)[90:]   # from near the peak: short records carry signal
    # the source on a tile corner (padded node (128, 8) when the grid reaches it),
    # receivers along a row and a column that cross tile edges
    sx, sz = min(128, w.nx + 2 * w.nb - 1), min(8, w.nz + 2 * w.nb - 1)
    src = np.array([sx, 0, sz], np.int32)
    xs = np.arange(0, w.nx + 2 * w.nb, 7)
    zs = np.arange(0, w.nz + 2 * w.nb, 5)
    rec = np.concatenate([np.stack([xs, 0 * xs, np.full_like(xs, min(15, w.nz + 2 * w.nb - 1))], 1),
                          np.stack([np.full_like(zs, min(127, w.nx + 2 * w.nb - 1)), 0 * zs, zs], 1)]).astype(np.int32)
    one = _run(R, monkeypatch, False, w, v, src, rec, wav)
    two = _run(R, monkeypatch, True, w, v, src, rec, wav)
    for k in one:
        assert np.array_equal(one[k], two[k]), k
    o = oracle_shot(w, v, src, rec, wav)
    assert rel(two["seis"], o["seis"]) <= TOL
    assert rel(two["last"], o["last"]) <= TOL
    if nt >= 100:   # after 3 steps the integrals are ~1e-26: nothing to compare against
        assert rel(two["num"], o["num"]) <= TOL and rel(two["den"], o["den"]) <= TOL


def test_two_levels_per_launch_fwi_gradient_unchanged(monkeypatch):
    import paper_2204_03380_gb300 as R
    from paper_2204_03380_gb300 import fwi
    from paper_2204_03380_gb300.fwi import fwi_misfit
    w = W.scaled(W.SMALL_2D, nx=60, nz=50, nb=10, nt=301, name="fwi_t")
    vt = W.three_layers(60, 50, (17, 35)).astype(np.float32)
    v0 = W.smooth_slowness(vt, 3.0).astype(np.float32) * np.float32(0.98)
    shots = [W.source_at(w, 20), W.source_at(w, 40)]
    rec = W.surface_line(w, step=2)
    g = R.make_grid(2, w.nx, 1, w.nz, w.nb, w.h, w.dt, w.nt)
    wt = torch.tensor(W.ricker(w.nt, w.dt, w.f_peak), dtype=torch.float32, device="cuda")
    rbc = (w.v_lo, w.v_hi, w.v_max, w.rbc_seed)
    grads = []
    for temporal in (False, True):
        if temporal:
            monkeypatch.setenv("RBC_TEMPORAL", "2")
        else:
            monkeypatch.delenv("RBC_TEMPORAL", raising=False)
        fwi.release_contexts()  # fresh contexts read the setting
        a = torch.empty(g.padded, dtype=torch.float32, device="cuda")
        R.rbc_build_velocity(g, torch.tensor(vt, device="cuda"), *rbc[:3], rbc[3], 0, None, a)
        ctx = R.rbc_create(g, a)
        dobs = []
        for s in shots:
            d = torch.empty((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
            R.rbc_model(ctx, s, wt, rec, d)
            dobs.append(d)
        R.rbc_destroy(ctx)
        v = torch.tensor(v0, device="cuda", requires_grad=True)
        J = fwi_misfit(v, g, shots, wt, rec, dobs, rbc)
        J.backward()
        grads.append((float(J.detach()), v.grad.cpu().numpy()))
    fwi.release_contexts()
    # the shots run concurrently and their sums are accumulated by atomic adds,
    # whose order (and so the last bits) may differ from run to run
    assert grads[1][0] == pytest.approx(grads[0][0], rel=1e-6)
    assert rel(grads[1][1], grads[0][1]) <= 1e-6
