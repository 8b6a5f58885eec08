"""The learned denoiser end to end: images from the RTM pipeline (K random
boundary realizations per model, via the batched path), training by the
project's own kernels, and the gain of the trained network over the method
without it (a single realization), measured against the K-stack on held-out
models."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _set(M, n=96, nb=24, nt=620, K=16, S=4, seed=0):
    import paper_2204_03380_gb300 as R
    from paper_2204_03380_gb300 import denoise as D
    w = W.scaled(W.SMALL_2D, nx=n, nz=n, nb=nb, nt=nt, name="denoise")
    vt = [W.faulted_layers(n, n, seed + m, 1500.0, 4000.0, nlayers=8, nfaults=2) for m in range(M)]
    vm = [W.smooth_slowness(v, 4.0) for v in vt]
    g = R.make_grid(2, n, 1, n, nb, w.h, w.dt, nt)
    shots = [W.source_at(w, int(x)) for x in np.linspace(n / (2 * S), n - n / (2 * S), S).astype(int)]
    rec = W.surface_line(w)
    return D.rtm_realizations(R, g, vt, vm, K, shots, rec, W.ricker(nt, w.dt, w.f_peak), (1500.0, 4000.0, 4000.0))


def test_stacking_reduces_the_random_boundary_noise():
    from paper_2204_03380_gb300 import denoise as D
    iset = _set(3)
    s = iset.stack
    half = iset.images[:, :8].mean(dim=1)
    # the realizations differ, and their mean moves towards the full stack
    assert D.rel_l2(iset.single, s) > 1e-2
    assert D.rel_l2(half, s) < D.rel_l2(iset.single, s)


def test_trained_network_beats_a_single_realization_on_held_out_models():
    from paper_2204_03380_gb300 import denoise as D
    train = _set(48, seed=0)
    test = _set(8, seed=5000)
    x, t, _ = D.normalized_pairs(train)
    x = torch.cat([x, x.flip(-1)])          # mirror augmentation
    t = torch.cat([t, t.flip(-1)])
    net = D.Denoiser(seed=1)
    l1 = net.fit(x, t, steps=1200, batch=16, lr=2e-3, seed=0)
    net.fit(x, t, steps=600, batch=16, lr=5e-4, seed=1)
    l3 = net.fit(x, t, steps=600, batch=16, lr=1e-4, seed=2)
    assert l3[-50:].mean() < l1[:20].mean()
    xs, ts, _ = D.normalized_pairs(test)
    e_single = D.rel_l2(xs, ts)
    e_net = D.rel_l2(net(xs), ts)
    print(f"held-out rel L2 to the 16-stack: single realization {e_single:.4f}, network {e_net:.4f}")
    assert e_net < 0.85 * e_single
