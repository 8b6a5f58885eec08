"""The denoiser's tensor-core kernels (rbc_cnn_*) against the FP64 oracle
(oracle/cnn.py, pinned by finite differences).  The oracle gets the GPU's
bf16-rounded parameters and inputs; hidden activations are bf16 on the GPU,
so the bar is relative L2 <= 1e-2 (forward) and <= 3e-2 (gradient)."""
import numpy as np
import pytest

from oracle import cnn
from rtm_cases import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("shape", [(2, 16, 32), (3, 37, 70), (2, 45, 300), (1, 9, 253)])
def test_cnn_forward_and_gradient_match_oracle(shape):
    import paper_2204_03380_gb300 as R
    rng = np.random.default_rng(sum(shape))
    p = cnn.init_params(4)
    p[-(9 * 32 + 1):] = rng.normal(0, 0.05, 9 * 32 + 1)
    p = bf16(p)
    x = bf16(rng.standard_normal(shape))
    t = rng.standard_normal(shape)
    y_o, cache = cnn.forward(p, x)
    g_o = cnn.backward(p, cache, 2 * (y_o - t) / y_o.size)
    dev = "cuda"
    P = torch.tensor(p, dtype=torch.float32, device=dev)
    X = torch.tensor(x, dtype=torch.float32, device=dev)
    T = torch.tensor(t, dtype=torch.float32, device=dev)
    Y = torch.empty_like(X)
    ws = torch.empty(R.rbc_cnn_workspace_bytes(*shape), dtype=torch.uint8, device=dev)
    R.rbc_cnn_forward(P, X, Y, ws)
    dY = torch.empty_like(X)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    R.rbc_cnn_mse(Y, T, dY, loss)
    G = torch.zeros_like(P)
    R.rbc_cnn_backward(P, dY, G, ws)
    torch.cuda.synchronize()
    # inference: the first layer built inside the second layer's kernel, the
    # same operations as the training forward, so the same bits
    Yi = torch.full_like(X, float("nan"))
    wsi = torch.empty_like(ws)
    R.rbc_cnn_infer(P, X, Yi, wsi)
    torch.cuda.synchronize()
    assert torch.equal(Yi, Y)
    assert R.rbc_cnn_param_count() == p.size
    assert rel(Y.cpu().numpy(), y_o) <= 1e-2
    assert float(loss) == pytest.approx(cnn.mse(y_o, t), rel=2e-2)
    assert rel(G.cpu().numpy(), g_o) <= 3e-2, rel(G.cpu().numpy(), g_o)
    # every layer's block on its own (the one-channel end layers have their
    # own weight-gradient kernel, and their blocks are small in the whole)
    for l, ((Wg, bg), (Wo, bo)) in enumerate(zip(cnn.split(G.cpu().numpy()), cnn.split(g_o))):
        assert rel(Wg, Wo) <= 3e-2, (l + 1, "W", rel(Wg, Wo))
        if bo.size > 1:
            assert rel(bg, bo) <= 3e-2, (l + 1, "b", rel(bg, bo))
    # db5 is the sum of dL/dy over the batch: the GPU sums the values rounded
    # to bf16 (relative error <= 2^-8 each)
    d = dY.double().cpu()
    assert abs(float(G[-1]) - float(d.sum())) <= 2.0 ** -8 * float(d.abs().sum())


def test_cnn_adam_steps_reduce_the_loss():
    import paper_2204_03380_gb300 as R
    rng = np.random.default_rng(9)
    dev = "cuda"
    x = rng.standard_normal((4, 32, 64))
    k = np.ones((3, 3)) / 9.0
    from scipy.signal import correlate2d
    t = np.stack([correlate2d(xi, k, mode="same") for xi in x])     # learn a smoothing
    P = torch.tensor(cnn.init_params(5), dtype=torch.float32, device=dev)
    X = torch.tensor(x, dtype=torch.float32, device=dev)
    T = torch.tensor(t, dtype=torch.float32, device=dev)
    Y, dY = torch.empty_like(X), torch.empty_like(X)
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    ws = torch.empty(R.rbc_cnn_workspace_bytes(*x.shape), dtype=torch.uint8, device=dev)
    losses = []
    for step in range(1, 61):
        G = torch.zeros_like(P)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        R.rbc_cnn_forward(P, X, Y, ws)
        R.rbc_cnn_mse(Y, T, dY, loss)
        R.rbc_cnn_backward(P, dY, G, ws)
        R.rbc_cnn_adam(P, G, M, V, 2e-3, step)
        losses.append(float(loss))
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_cnn_adam_matches_the_oracle_step_by_step():
    # rbc_cnn_adam against oracle.cnn.adam (Kingma & Ba 2015, Algorithm 1) on
    # the same fp32 gradients: parameters and both moments after every step,
    # element by element; the hyper-parameters are the fp32 values the kernel
    # receives.  Gradients mix magnitudes (down to eps) and exact zeros.
    import paper_2204_03380_gb300 as R
    rng = np.random.default_rng(11)
    n = R.rbc_cnn_param_count()
    lr, b1, b2, eps = (float(np.float32(x)) for x in (3e-3, 0.9, 0.999, 1e-8))
    p = (0.05 * rng.standard_normal(n)).astype(np.float32).astype(np.float64)   # weights of the trained scale
    m = np.zeros(n)
    v = np.zeros(n)
    dev = "cuda"
    P = torch.tensor(p, dtype=torch.float32, device=dev)
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    p0 = p.copy()
    for step in range(1, 9):
        g = (rng.standard_normal(n) * 10.0 ** rng.integers(-8, 1, n)).astype(np.float32)
        g[rng.random(n) < 0.05] = 0.0
        G = torch.tensor(g, device=dev)
        R.rbc_cnn_adam(P, G, M, V, lr, step, b1, b2, eps)
        p, m, v = cnn.adam(p, g.astype(np.float64), m, v, lr, b1, b2, eps, step)
        torch.cuda.synchronize()
        assert rel(M.cpu().numpy(), m) <= 1e-6
        assert rel(V.cpu().numpy(), v) <= 1e-6
        # the accumulated update (the parameters themselves hide it behind |p|)
        assert rel(P.cpu().numpy().astype(np.float64) - p0, p - p0) <= 1e-5
