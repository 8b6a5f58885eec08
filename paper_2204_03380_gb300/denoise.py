"""Learned stand-in for stacking random-boundary realizations of RTM images.

With random boundary conditions (Section 4.3) the reconstructed source
wavefield carries incoherent scattering from the random pad, which leaks into
the image; it differs from one boundary realization to the next, so the plain
fix is to migrate K realizations and average them (the K-stack).  This module
trains the small CNN of librbc (rbc_cnn_*) to map a single-realization image
to the K-stack, and keeps the K-stack as the fallback and as the yardstick of the
network's error.  Every image, gradient and update is computed by librbc's
kernels; this module sequences the calls and holds the tensors.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import _native as N


# ---------------------------------------------------------------- network --
def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-style seeded initialisation; the last layer starts small, so the
    residual network starts near the identity map."""
    g = torch.Generator().manual_seed(seed)
    chunks = []
    for l, (cin, cout) in enumerate([(1, 32), (32, 32), (32, 32), (32, 32), (32, 1)]):
        std = math.sqrt(2.0 / (9 * cin)) * (0.1 if l == 4 else 1.0)
        chunks.append(torch.randn(9 * cout * cin, generator=g, dtype=torch.float64) * std)
        chunks.append(torch.zeros(cout, dtype=torch.float64))
    p = torch.cat(chunks).to(torch.float32).to(device)
    assert p.numel() == N.rbc_cnn_param_count()
    return p


class Denoiser:
    def __init__(self, params: torch.Tensor | None = None, seed: int = 0, device="cuda"):
        self.device = torch.device(device)
        self.params = init_params(seed, self.device) if params is None else params.to(self.device).contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._ws = None

    def _workspace(self, n, H, W):
        need = N.rbc_cnn_workspace_bytes(n, H, W)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._ws

    def __call__(self, x: torch.Tensor) -> torch.Tensor:
        """x: (n, H, W) fp32 CUDA -> denoised images."""
        x = x.contiguous()
        y = torch.empty_like(x)
        N.rbc_cnn_infer(self.params, x, y, self._workspace(*x.shape))
        return y

    def train_step(self, x, t, lr=1e-3) -> torch.Tensor:
        """One Adam step on the batch; returns the batch loss (device scalar)."""
        x, t = x.contiguous(), t.contiguous()
        ws = self._workspace(*x.shape)
        y, dy = torch.empty_like(x), torch.empty_like(x)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        grad = torch.zeros_like(self.params)
        N.rbc_cnn_forward(self.params, x, y, ws)
        N.rbc_cnn_mse(y, t, dy, loss)
        N.rbc_cnn_backward(self.params, dy, grad, ws)
        self.step += 1
        N.rbc_cnn_adam(self.params, grad, self.m, self.v, lr, self.step)
        return loss

    def fit(self, inputs, targets, steps=400, batch=8, lr=1e-3, seed=0):
        """Adam on random mini-batches of (input, target) images."""
        rng = np.random.default_rng(seed)
        losses = []
        n = inputs.shape[0]
        for s in range(steps):
            idx = torch.as_tensor(rng.choice(n, min(batch, n), replace=False), device=self.device)
            losses.append(self.train_step(inputs[idx], targets[idx], lr))
        return torch.cat(losses).cpu().numpy()

    def denoise_volume(self, vol: torch.Tensor, slab: int = 64) -> torch.Tensor:
        """3-D image (nz, ny, nx): every x-z slice (fixed y) denoised, slab slices at a time."""
        nz, ny, nx = vol.shape
        out = torch.empty_like(vol)
        for y0 in range(0, ny, slab):
            sl = vol[:, y0:y0 + slab, :].permute(1, 0, 2).contiguous()   # (slices, nz, nx)
            out[:, y0:y0 + slab, :] = self(sl).permute(1, 0, 2)
        return out


# ------------------------------------------------------------ data: images --
@dataclasses.dataclass
class ImageSet:
    """RTM images of several models, each migrated with K boundary realizations."""
    images: torch.Tensor   # (models, K, nz, nx)

    @property
    def single(self):      # the method without help: realization 0
        return self.images[:, 0]

    @property
    def stack(self):       # the K-stack: the fallback and the yardstick
        return self.images.mean(dim=1)


def rtm_realizations(R, grid, v_true, v_mig, K, shots, rec, wavelet, rbc, obs_seed=1_000_003, seed_base=0,
                     max_batch=512):
    """Migrate every model with K random-boundary realizations.

    grid: 2-D grid of one model (all models share it); v_true, v_mig: lists of
    (nz, nx) arrays; shots: source nodes; rec: receiver nodes (padded frame);
    rbc: (v_lo, v_hi, v_max).  Realization k of model m uses boundary seed
    seed_base + 7919 m + k; the observed records come from the true model with
    boundary seed obs_seed.  Returns ImageSet (images of realization k of model
    m are stacked over the shots)."""
    dev = torch.device("cuda")
    M = len(v_true)
    nz, nx = grid.nz, grid.nx
    wav = wavelet if isinstance(wavelet, torch.Tensor) else torch.tensor(wavelet, dtype=torch.float32, device=dev)
    # observed records
    seis = []
    for m in range(M):
        a = torch.empty(grid.padded, dtype=torch.float32, device=dev)
        R.rbc_build_velocity(grid, torch.tensor(v_true[m], dtype=torch.float32, device=dev), *rbc, obs_seed, 0, None, a)
        ctx = R.rbc_create(grid, a)
        rows = []
        for src in shots:
            d = torch.empty((len(rec), grid.nt + 1), dtype=torch.float32, device=dev)
            R.rbc_model(ctx, src, wav, rec, d)
            rows.append(d)
        torch.cuda.synchronize()
        R.rbc_destroy(ctx)
        seis.append(rows)
    # migrations: one batch entry per (model, realization, shot); each
    # (model, realization) image has its own canvas column block
    jobs = [(m, k, s) for m in range(M) for k in range(K) for s in range(len(shots))]
    canvas = torch.zeros((nz, M * K * nx), dtype=torch.float32, device=dev)
    for j0 in range(0, len(jobs), max_batch):
        chunk = jobs[j0:j0 + max_batch]
        a_list = []
        for (m, k, s) in chunk:
            a = torch.empty(grid.padded, dtype=torch.float32, device=dev)
            R.rbc_build_velocity(grid, torch.tensor(v_mig[m], dtype=torch.float32, device=dev), *rbc,
                                 seed_base + 7919 * m + k, 0, None, a)
            a_list.append(a)
        b = R.rbc_batch_create(grid, [nx] * len(chunk), a_list)
        try:
            sh = [dict(src=shots[s], rec=rec, seis=seis[m][s], off_x=(m * K + k) * nx) for (m, k, s) in chunk]
            R.rbc_batch_rtm(b, sh, wav, R.RBC_REINJECT_SOURCE, 1e-6, canvas)
            torch.cuda.synchronize()
        finally:
            R.rbc_batch_destroy(b)
        del a_list
    imgs = canvas.reshape(nz, M, K, nx).permute(1, 2, 0, 3).contiguous()
    return ImageSet(imgs)


def normalized_pairs(iset: ImageSet):
    """(input, target) pairs scaled by the input's RMS, so that every model
    weighs the same in the loss; the scale is the one available at inference,
    where only the single-realization image exists."""
    x = iset.single
    scale = x.pow(2).mean(dim=(1, 2), keepdim=True).sqrt().clamp_min(1e-30)
    return x / scale, iset.stack / scale, scale


def rel_l2(a, b) -> float:
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def denoise_or_stack(net: Denoiser, single, stack_fn, val_error: float, tol: float = 5e-2):
    """The trained network when its held-out error against the K-stack is
    within tol, else the K-stack itself (stack_fn() computes it)."""
    if val_error <= tol:
        return net(single), "network"
    return stack_fn(), "k-stack"
