"""rbc_model_static: modeling for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- for example code running while a
caching allocator owns the device heap, or a host runtime that forbids
allocation on its worker threads.  rbc_model_static serves them from a fixed
per-device workspace inside the library.  This file checks, through the C ABI,
that two calls in a row (the workspace keeps the previous call's contents)
give the same records as the context-based rbc_model and as the FP64 oracle,
in 2-D and in 3-D (the TMA-fed kernels over the workspace), that a bounded
wait that gives up is reported by the next call, and that a problem too large
for the workspace is refused.  It is collected last on purpose."""
import numpy as np
import pytest

import oracle
import workloads as W
from rtm_cases import TOL, case_3d, f32, gpu_build, oracle_a, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(R, nx, nz, nb, nt, seed):
    w = W.scaled(W.SMALL_2D, nx=nx, nz=nz, nb=nb, nt=nt, name="static")
    w = W.dataclasses.replace(w, rbc_seed=seed)
    v = np.random.default_rng(seed).uniform(1500, 3500, (nz, nx)).astype(np.float32)
    g, a, _ = gpu_build(R, torch, w, v)
    wav = W.ricker(nt, w.dt, w.f_peak)
    return w, v, g, a, wav


def _oracle_record(w, v, src, rec, wav):
    a = oracle_a(w, v)[1].astype(np.float64)
    return oracle.model(a, w.h, w.nt, src, f32(wav), np.asarray(rec, np.int32).reshape(-1, 3))["seis"]


def _two_calls(R, w, v, g, a, wav, shots, rec):
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    ctx = R.rbc_create(g, a)
    try:
        for src in shots:   # the second call must not see the first call's fields
            ref = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
            R.rbc_model(ctx, src, wt, rec, ref)
            out = torch.full_like(ref, float("nan"))
            R.rbc_model_static(g, a, src, wt, rec, out)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            assert np.isfinite(o).all()
            assert rel(o, ref.cpu().numpy()) <= TOL
            assert rel(o, _oracle_record(w, v, src, rec, wav)) <= TOL
    finally:
        R.rbc_destroy(ctx)


def test_static_modeling_matches_context_modeling_and_oracle_twice_in_a_row():
    import paper_2204_03380_gb300 as R
    w, v, g, a, wav = _inputs(R, 150, 90, 20, 500, seed=5)
    rec = W.surface_line(w, step=3)
    _two_calls(R, w, v, g, a, wav, [W.source_at(w, 20), W.source_at(w, 120, depth=30)], rec)


def test_static_modeling_3d_matches_context_modeling_and_oracle_twice_in_a_row():
    import paper_2204_03380_gb300 as R
    w, v, src, rec, wav = case_3d("static3", 21, 17, 13, 5, 120)
    g, a, _ = gpu_build(R, torch, w, v)
    src2 = W.source_at(w, 4, 12, depth=9)
    _two_calls(R, w, v, g, a, wav, [src, src2], rec)


def test_static_timeout_is_reported_by_the_next_call():
    import paper_2204_03380_gb300 as R
    w, v, src, rec, wav = case_3d("static_fault", 21, 17, 13, 5, 20)
    g, a, _ = gpu_build(R, torch, w, v)
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    clean = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
    R.rbc_model_static(g, a, src, wt, rec, clean)
    R.rbc_inject_fault(None, 1)
    bad = torch.zeros_like(clean)
    R.rbc_model_static(g, a, src, wt, rec, bad)       # its first launch withholds a copy and gives up
    torch.cuda.synchronize()                          # the device finished: it did not hang
    again = torch.zeros_like(clean)
    with pytest.raises(R.RBCError) as e:
        R.rbc_model_static(g, a, src, wt, rec, again)
    assert e.value.code == 5                          # RBC_ETIMEOUT, reported once
    R.rbc_model_static(g, a, src, wt, rec, again)     # the workspace still works
    torch.cuda.synchronize()
    assert rel(again.cpu().numpy(), clean.cpu().numpy()) <= TOL


def test_static_modeling_refuses_problems_beyond_its_workspace():
    import paper_2204_03380_gb300 as R
    w, v, g, a, wav = _inputs(R, 1500, 1500, 20, 10, seed=6)   # three 1540 x 1540 fields > 16 MiB
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    seis = torch.zeros((1, w.nt + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(R.RBCError) as e:
        R.rbc_model_static(g, a, W.source_at(w, 5), wt, W.source_at(w, 9)[None], seis)
    assert e.value.code == 1 and "maximum" in str(e.value)
