"""Host logic of the Python drivers above the ABI, on CPU tensors (no kernels
run): the denoiser's training-pair scaling, error measure and fallback to the
K-stack, and the FWI function's shots in flight."""
import pytest

torch = pytest.importorskip("torch")

from paper_2204_03380_gb300 import denoise as D  # noqa: E402


def _set(models=3, K=4, n=6, seed=0):
    g = torch.Generator().manual_seed(seed)
    return D.ImageSet(torch.randn((models, K, n, n), generator=g, dtype=torch.float64))


def test_single_and_stack_views():
    s = _set()
    assert torch.equal(s.single, s.images[:, 0])
    assert torch.allclose(s.stack, s.images.mean(dim=1))


def test_pairs_are_scaled_by_the_input_rms_only():
    s = _set()
    x, t, scale = D.normalized_pairs(s)
    # every input has unit RMS; the target carries the same per-model factor
    assert torch.allclose(x.pow(2).mean(dim=(1, 2)), torch.ones(3, dtype=torch.float64))
    assert torch.allclose(t * scale, s.stack) and torch.allclose(x * scale, s.single)
    # scaling a model's realizations leaves its pair unchanged
    s2 = D.ImageSet(s.images.clone())
    s2.images[1] *= 7.0
    x2, t2, _ = D.normalized_pairs(s2)
    assert torch.allclose(x2, x) and torch.allclose(t2, t)


def test_rel_l2():
    b = torch.tensor([3.0, 4.0])
    assert D.rel_l2(b, b) == 0.0
    assert D.rel_l2(torch.zeros(2), b) == pytest.approx(1.0)
    assert D.rel_l2(b * 1.1, b) == pytest.approx(0.1)


def test_fallback_to_the_k_stack():
    calls = []

    def net(x):
        return x + 1

    def stack_fn():
        calls.append(1)
        return "stack"

    single = torch.zeros(2)
    out, which = D.denoise_or_stack(net, single, stack_fn, val_error=0.04)
    assert which == "network" and torch.equal(out, single + 1) and not calls
    out, which = D.denoise_or_stack(net, single, stack_fn, val_error=0.06)
    assert which == "k-stack" and out == "stack" and calls == [1]
    assert D.denoise_or_stack(net, single, stack_fn, val_error=0.05)[1] == "network"


def test_fwi_shots_in_flight():
    """The FWI autograd function runs several shots at once only while their
    contexts' fields stay within the pool's L2-sized budget."""
    import paper_2204_03380_gb300 as R
    from paper_2204_03380_gb300 import fwi
    small = R.make_grid(2, 300, 1, 300, 50, 10.0, 1e-3, 1000)      # 0.64 MB per field
    assert fwi.shot_streams(small, 4) == 4 and fwi.shot_streams(small, 2) == 2 and fwi.shot_streams(small, 9) == 4
    survey = R.make_grid(2, 2301, 1, 751, 60, 4.0, 4e-4, 12500)   # 8.4 MB per field
    assert fwi.shot_streams(survey, 8) == 1
    assert fwi._grid_key(small) != fwi._grid_key(survey)
    assert fwi._grid_key(small) == fwi._grid_key(R.make_grid(2, 300, 1, 300, 50, 10.0, 1e-3, 1000))
