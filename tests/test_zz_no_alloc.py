"""rbc_model_static: modeling for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- for example code running while a
caching allocator owns the device heap, or a host runtime that forbids
allocation on its worker threads.  rbc_model_static serves them from a fixed
per-device workspace inside the library.  This file checks, through the C ABI,
that two calls in a row (the workspace keeps the previous call's contents)
give the same records as the context-based rbc_model, and that a problem too
large for the workspace is refused.  It is collected last on purpose."""
import numpy as np
import pytest

import workloads as W
from rtm_cases import TOL, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(R, nx, nz, nb, nt, seed):
    w = W.scaled(W.SMALL_2D, nx=nx, nz=nz, nb=nb, nt=nt, name="static")
    g = R.make_grid(2, w.nx, 1, w.nz, w.nb, w.h, w.dt, w.nt)
    v = torch.tensor(np.random.default_rng(seed).uniform(1500, 3500, (nz, nx)), dtype=torch.float32,
                     device="cuda")
    a = torch.empty(g.padded, dtype=torch.float32, device="cuda")
    R.rbc_build_velocity(g, v, w.v_lo, w.v_hi, w.v_max, seed, 0, None, a)
    wav = torch.tensor(W.ricker(nt, w.dt, w.f_peak), dtype=torch.float32, device="cuda")
    return w, g, a, wav


def test_static_modeling_matches_context_modeling_twice_in_a_row():
    import paper_2204_03380_gb300 as R
    w, g, a, wav = _inputs(R, 150, 90, 20, 500, seed=5)
    rec = W.surface_line(w, step=3)
    shots = [W.source_at(w, 20), W.source_at(w, 120, depth=30)]
    ctx = R.rbc_create(g, a)
    try:
        for src in shots:   # the second call must not see the first call's fields
            ref = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
            R.rbc_model(ctx, src, wav, rec, ref)
            out = torch.full_like(ref, float("nan"))
            R.rbc_model_static(g, a, src, wav, rec, out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= TOL
    finally:
        R.rbc_destroy(ctx)


def test_static_modeling_refuses_problems_beyond_its_workspace():
    import paper_2204_03380_gb300 as R
    w, g, a, wav = _inputs(R, 1500, 1500, 20, 10, seed=6)   # three 1540 x 1540 fields > 16 MiB
    seis = torch.zeros((1, w.nt + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(R.RBCError) as e:
        R.rbc_model_static(g, a, W.source_at(w, 5), wav, W.source_at(w, 9)[None], seis)
    assert e.value.code == 1 and "maximum" in str(e.value)
