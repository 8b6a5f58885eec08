"""FWI misfit and velocity gradient as a torch.autograd.Function.

forward(v_int): builds the padded coefficient with the random boundary
(rbc_build_velocity), then for every shot rbc_fwi_forward (modeling, residual,
misfit) and keeps only the residual and the two last panels of the shot.
backward: for every shot rbc_fwi_backward rebuilds the source wavefield
backwards from those panels -- the random boundary makes the recursion
reversible, so nothing is stored or checkpointed -- while it runs the exact
discrete adjoint, and accumulates dJ/dv on the interior.  All arithmetic runs
in librbc's kernels; this module only sequences the calls.

The shots are independent, so they run on a small pool of contexts, one CUDA
stream each, kept per grid across calls: a context's coefficient is replaced
with rbc_set_coef (no allocation, the captured time-loop graphs are reused),
and small grids, which fill only part of the GPU per launch, get several shots
in flight at once.  The misfit and the gradient are accumulated by the
kernels' atomic adds, so the streams share them.
"""
from __future__ import annotations

import torch

from . import _native as N

# contexts in flight at once: up to MAX_STREAMS, while their fields (seven per
# context) stay within POOL_BYTES, so that the shots in flight share L2 instead
# of evicting one another
MAX_STREAMS = 4
POOL_BYTES = 64 << 20

_POOL: dict = {}


def _grid_key(grid):
    return tuple(getattr(grid, f) for f, _ in grid._fields_)


def shot_streams(grid, nshots):
    """Shots in flight at once for this grid: at most MAX_STREAMS, and no more
    than the contexts whose seven fields fit in POOL_BYTES."""
    nodes = 1
    for n in grid.padded:
        nodes *= n
    fit = max(1, POOL_BYTES // (7 * 4 * nodes))
    return max(1, min(nshots, MAX_STREAMS, fit))


def _pool(grid, a, n, device):
    """n (context, stream) pairs for this grid on this device."""
    key = (_grid_key(grid), device.index)
    pool = _POOL.setdefault(key, [])
    while len(pool) < n:
        pool.append((N.rbc_create(grid, a), torch.cuda.Stream(device)))
    return pool[:n]


def release_contexts():
    """Destroy the pooled contexts (after the device work that uses them)."""
    torch.cuda.synchronize()
    for pool in _POOL.values():
        for ctx, _ in pool:
            N.rbc_destroy(ctx)
    _POOL.clear()


def _fan_out(grid, a, nshots, device, check):
    """Contexts and streams for nshots shots, each holding coefficient a
    (checked once when check); the streams start after the current stream's
    work so far."""
    main = torch.cuda.current_stream(device)
    pool = _pool(grid, a, shot_streams(grid, nshots), device)
    start = torch.cuda.Event()
    start.record(main)
    for k, (ctx, s) in enumerate(pool):
        s.wait_event(start)
        N.rbc_set_coef(ctx, grid, a, check and k == 0, s)   # ordered after the context's earlier work
    return main, pool


def _join(main, pool, tensors):
    """The current stream waits for every stream of the pool; tensors the
    streams used are marked for the caching allocator."""
    for _, s in pool:
        for t in tensors:
            t.record_stream(s)
        done = torch.cuda.Event()
        done.record(s)
        main.wait_event(done)


class FWIMisfit(torch.autograd.Function):
    @staticmethod
    def forward(fctx, v_int, grid, shots, wavelet, rec, dobs, rbc):
        """v_int: interior velocity (nz, nx) fp32 CUDA; shots: list of source
        nodes; dobs: list of (nrec, nt+1) records; rbc: (v_lo, v_hi, v_max, seed)."""
        dev = v_int.device
        a = torch.empty(grid.padded, dtype=torch.float32, device=dev)
        N.rbc_build_velocity(grid, v_int.detach().contiguous(), *rbc[:3], rbc[3], 0, None, a)
        misfit = torch.zeros(1, dtype=torch.float64, device=dev)
        resids = [torch.empty_like(d) for d in dobs]
        panels = [torch.empty((2,) + tuple(grid.padded), dtype=torch.float32, device=dev) for _ in shots]
        main, pool = _fan_out(grid, a, len(shots), dev, check=True)
        for i, (src, d) in enumerate(zip(shots, dobs)):
            ctx, s = pool[i % len(pool)]
            N.rbc_fwi_forward(ctx, src, wavelet, rec, d, resids[i], misfit, panels[i], stream=s)
        _join(main, pool, [a, misfit, wavelet, *dobs, *resids, *panels])
        fctx.grid, fctx.shots, fctx.rec = grid, shots, rec
        fctx.save_for_backward(a, wavelet, *resids, *panels)
        return misfit.to(torch.float32).reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        saved = fctx.saved_tensors
        a, wavelet = saved[0], saved[1]
        n = len(fctx.shots)
        resids, panels = saved[2:2 + n], saved[2 + n:2 + 2 * n]
        grid = fctx.grid
        g = torch.zeros(grid.interior, dtype=torch.float32, device=wavelet.device)
        # the coefficient of this forward call (another call may have replaced it since)
        main, pool = _fan_out(grid, a, n, wavelet.device, check=False)
        for i, (src, r, p) in enumerate(zip(fctx.shots, resids, panels)):
            ctx, s = pool[i % len(pool)]
            N.rbc_fwi_backward(ctx, src, wavelet, fctx.rec, r, p, g, stream=s)
        _join(main, pool, [a, g, wavelet, *resids, *panels])
        return g * grad_out.to(g.dtype), None, None, None, None, None, None


def fwi_misfit(v_int, grid, shots, wavelet, rec, dobs, rbc):
    """J(v) = sum over shots of 1/2 ||record - dobs||^2, differentiable in v_int."""
    return FWIMisfit.apply(v_int, grid, shots, wavelet, rec, dobs, rbc)
