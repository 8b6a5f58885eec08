"""Batched RTM of uneven-aperture shots (rbc_batch_*) against the single-shot
path and against the FP64 oracle's stacked image."""
import numpy as np
import pytest

import oracle
import workloads as W
from rtm_cases import ILLUM, TOL, f32, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small_batch():
    w = W.scaled(W.BATCH_2D, nx=300, nz=50, nb=10, nt=400, name="batch_small")
    w = W.dataclasses.replace(w, nshots=5)
    inp = W.batch_2d_inputs(w, wmin=40, wmax=130, rec_step=3)
    return w, inp


def _shot_grid(R, w, width):
    return R.make_grid(2, width, 1, w.nz, w.nb, w.h, w.dt, w.nt)


def _window(v, off, width):
    return np.ascontiguousarray(v[:, off:off + width])


# every forward kernel the autotuner can pick (0 = the streaming kernel) and
# every reverse kernel (1 or 2 rows per warp, 0 = streaming, 3 = shared-memory
# tiles), forced one pair at a time, and the tuner's own choice;
# one group of all shots, one shot per group (0.3 MB) and groups of two or
# three shots (1.5 MB)
@pytest.mark.parametrize("tiles,l2mb,groups", [(None, None, 1), ("0,0", None, 1), ("4,2", None, 1),
                                               (None, "0.3", 5), ("0,0", "1.5", None), ("1,1", "0", 1),
                                               ("2,3", None, 1), ("2,3", "0.3", 5)])
def test_batch_matches_single_shots_and_oracle(tiles, l2mb, groups, monkeypatch):
    import paper_2204_03380_gb300 as R
    if tiles is not None:
        monkeypatch.setenv("RBC_BATCH_TILES", tiles)
    if l2mb is not None:
        monkeypatch.setenv("RBC_BATCH_L2MB", l2mb)
    w, inp = _small_batch()
    dev = "cuda"
    wav = torch.tensor(inp["wavelet"], dtype=torch.float32, device=dev)
    a_true, a_mig, seis = [], [], []
    for sh in inp["shots"]:
        g = _shot_grid(R, w, sh["width"])
        for v, out in ((inp["v_true"], a_true), (inp["v_mig"], a_mig)):
            a = torch.empty(g.padded, dtype=torch.float32, device=dev)
            vw = torch.tensor(_window(v, sh["off_x"], sh["width"]), dtype=torch.float32, device=dev)
            R.rbc_build_velocity(g, vw, w.v_lo, w.v_hi, w.v_max, w.rbc_seed, 0, None, a)
            out.append(a)
        ctx = R.rbc_create(g, a_true[-1])
        d = torch.empty((len(sh["rec"]), w.nt + 1), dtype=torch.float32, device=dev)
        R.rbc_model(ctx, sh["src"], wav, sh["rec"], d)
        R.rbc_destroy(ctx)
        seis.append(d)
    # batched path
    b = R.rbc_batch_create(_shot_grid(R, w, 1), [sh["width"] for sh in inp["shots"]], a_mig)
    info = R.rbc_batch_info(b)
    assert info["rows_fwd"] in (0, 1, 2, 4) and info["rows_rev"] in (0, 1, 2, 3)
    if tiles is not None:
        assert [info["rows_fwd"], info["rows_rev"]] == [int(v) for v in tiles.split(",")]
    if groups is not None:
        assert info["groups"] == groups
    else:
        assert 1 < info["groups"] < len(inp["shots"])
    img_b = torch.zeros((w.nz, w.nx), dtype=torch.float32, device=dev)
    shots = [dict(src=sh["src"], rec=sh["rec"], seis=d, off_x=sh["off_x"]) for sh, d in zip(inp["shots"], seis)]
    R.rbc_batch_rtm(b, shots, wav, R.RBC_REINJECT_SOURCE, 1e-6, img_b)
    img_b2 = torch.zeros_like(img_b)
    R.rbc_batch_rtm(b, shots, wav, R.RBC_REINJECT_SOURCE, 1e-6, img_b2)   # graph replay
    torch.cuda.synchronize()
    R.rbc_batch_destroy(b)
    # single-shot path
    survey = R.make_grid(2, w.nx, 1, w.nz, w.nb, w.h, w.dt, w.nt)
    img_s = torch.zeros_like(img_b)
    for sh, a, d in zip(inp["shots"], a_mig, seis):
        g = _shot_grid(R, w, sh["width"])
        ctx = R.rbc_create(g, a)
        num = torch.zeros(g.interior, dtype=torch.float32, device=dev)
        den = torch.zeros_like(num)
        R.rbc_rtm_shot(ctx, sh["src"], wav, sh["rec"], d, R.RBC_REINJECT_SOURCE, num, den)
        R.rbc_image_stack(g, num, den, 1e-6, sh["off_x"], 0, survey, img_s)
        R.rbc_destroy(ctx)
    torch.cuda.synchronize()
    ib, ib2, isg = img_b.cpu().numpy(), img_b2.cpu().numpy(), img_s.cpu().numpy()
    assert rel(ib, isg) <= 1e-5 and rel(ib2, ib) <= 1e-6
    # oracle: per-shot image on the illuminated part, stacked
    ostack = np.zeros((w.nz, w.nx))
    mask = np.ones((w.nz, w.nx), bool)
    for sh, d in zip(inp["shots"], seis):
        ws = W.dataclasses.replace(w, nx=sh["width"])
        vp = oracle.rbc_velocity(f32(_window(inp["v_mig"], sh["off_x"], sh["width"])), w.nb, w.v_lo, w.v_hi,
                                 w.v_max, w.rbc_seed)
        a = oracle.coef(vp, w.dt, w.h)[1].astype(np.float64)
        r = oracle.rtm_shot(a, w.h, w.nt, sh["src"], f32(inp["wavelet"]), sh["rec"], d.cpu().numpy().astype(float),
                            w.nb, (ws.nx, 1, w.nz))
        img = oracle.image(r["num"], r["den"], 1e-6)
        oracle.stack(ostack, img, sh["off_x"])
        m = np.ones((w.nz, w.nx), bool)
        m[:, sh["off_x"]:sh["off_x"] + sh["width"]] = r["den"] >= ILLUM * r["den"].max()
        mask &= m
    assert mask.mean() > 0.3
    assert rel(ib[mask], ostack[mask]) <= TOL


def test_batch_rejects_bad_windows():
    import paper_2204_03380_gb300 as R
    w, inp = _small_batch()
    sh = inp["shots"][0]
    g = _shot_grid(R, w, sh["width"])
    a = torch.full(g.padded, 0.1, dtype=torch.float32, device="cuda")
    b = R.rbc_batch_create(g, [sh["width"]], [a])
    wav = torch.zeros(w.nt, dtype=torch.float32, device="cuda")
    img = torch.zeros((w.nz, 20), dtype=torch.float32, device="cuda")
    seis = torch.zeros((len(sh["rec"]), w.nt + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(R.RBCError) as e:
        R.rbc_batch_rtm(b, [dict(src=sh["src"], rec=sh["rec"], seis=seis, off_x=0)], wav,
                        R.RBC_REINJECT_SOURCE, 1e-6, img)
    assert e.value.code == 1
    R.rbc_batch_destroy(b)


def test_tiled_reverse_over_more_shots_than_one_launch_holds(monkeypatch):
    """18 shots in one group: the tiled reverse takes at most 16 shots' tile
    descriptors per launch, so each step is two launches (16 + 2 shots); the
    batched image equals the single-shot path's."""
    import paper_2204_03380_gb300 as R
    monkeypatch.setenv("RBC_BATCH_TILES", "2,3")
    w = W.scaled(W.BATCH_2D, nx=300, nz=40, nb=10, nt=150, name="batch_many")
    w = W.dataclasses.replace(w, nshots=18)
    inp = W.batch_2d_inputs(w, wmin=30, wmax=60, rec_step=3)
    dev = "cuda"
    wav = torch.tensor(inp["wavelet"], dtype=torch.float32, device=dev)
    a_mig, seis = [], []
    for sh in inp["shots"]:
        g = _shot_grid(R, w, sh["width"])
        at = torch.empty(g.padded, dtype=torch.float32, device=dev)
        R.rbc_build_velocity(g, torch.tensor(_window(inp["v_true"], sh["off_x"], sh["width"]), dtype=torch.float32,
                                             device=dev),
                             w.v_lo, w.v_hi, w.v_max, w.rbc_seed, 0, None, at)
        am = torch.empty_like(at)
        R.rbc_build_velocity(g, torch.tensor(_window(inp["v_mig"], sh["off_x"], sh["width"]), dtype=torch.float32,
                                             device=dev),
                             w.v_lo, w.v_hi, w.v_max, w.rbc_seed, 0, None, am)
        ctx = R.rbc_create(g, at)
        d = torch.empty((len(sh["rec"]), w.nt + 1), dtype=torch.float32, device=dev)
        R.rbc_model(ctx, sh["src"], wav, sh["rec"], d)
        R.rbc_destroy(ctx)
        a_mig.append(am)
        seis.append(d)
    b = R.rbc_batch_create(_shot_grid(R, w, 1), [sh["width"] for sh in inp["shots"]], a_mig)
    info = R.rbc_batch_info(b)
    assert info["rows_rev"] == 3 and info["groups"] == 1
    img_b = torch.zeros((w.nz, w.nx), dtype=torch.float32, device=dev)
    shots = [dict(src=sh["src"], rec=sh["rec"], seis=d, off_x=sh["off_x"]) for sh, d in zip(inp["shots"], seis)]
    R.rbc_batch_rtm(b, shots, wav, R.RBC_REINJECT_SOURCE, 1e-6, img_b)
    torch.cuda.synchronize()
    R.rbc_batch_destroy(b)
    survey = R.make_grid(2, w.nx, 1, w.nz, w.nb, w.h, w.dt, w.nt)
    img_s = torch.zeros_like(img_b)
    for sh, a, d in zip(inp["shots"], a_mig, seis):
        g = _shot_grid(R, w, sh["width"])
        ctx = R.rbc_create(g, a)
        num = torch.zeros(g.interior, dtype=torch.float32, device=dev)
        den = torch.zeros_like(num)
        R.rbc_rtm_shot(ctx, sh["src"], wav, sh["rec"], d, R.RBC_REINJECT_SOURCE, num, den)
        R.rbc_image_stack(g, num, den, 1e-6, sh["off_x"], 0, survey, img_s)
        R.rbc_destroy(ctx)
    torch.cuda.synchronize()
    assert float(img_s.abs().max()) > 0
    assert rel(img_b.cpu().numpy(), img_s.cpu().numpy()) <= 1e-5
