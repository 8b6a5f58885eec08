"""Failure detection without a GPU fault: a TMA plane copy that is never
issued makes a 3-D kernel's bounded mbarrier wait run out (about a second);
the kernel records it and returns, the next call reports RBC_ETIMEOUT, and
the context keeps working."""
import numpy as np
import pytest

from rtm_cases import TOL, case_3d, gpu_build, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_withheld_copy_times_out_and_the_context_recovers():
    import paper_2204_03380_gb300 as R
    w, v, src, rec, wav = case_3d("fault", 21, 17, 13, 5, 20)
    g, a, _ = gpu_build(R, torch, w, v)
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    ctx = R.rbc_create(g, a)
    try:
        clean = torch.zeros((len(rec), w.nt + 1), dtype=torch.float32, device="cuda")
        R.rbc_model(ctx, src, wt, rec, clean)
        R.rbc_inject_fault(ctx, 1)
        bad = torch.zeros_like(clean)
        R.rbc_model(ctx, src, wt, rec, bad)           # queued; its first launch gives up
        torch.cuda.synchronize()                      # the device finished: it did not hang
        again = torch.zeros_like(clean)
        with pytest.raises(R.RBCError) as e:
            R.rbc_model(ctx, src, wt, rec, again)
        assert e.value.code == 5                      # RBC_ETIMEOUT
        R.rbc_model(ctx, src, wt, rec, again)         # reported once; the context still works
        torch.cuda.synchronize()
        assert rel(again.cpu().numpy(), clean.cpu().numpy()) <= TOL
    finally:
        R.rbc_destroy(ctx)
