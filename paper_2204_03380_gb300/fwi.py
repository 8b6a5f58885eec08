"""FWI misfit and velocity gradient as a torch.autograd.Function.

forward(v_int): builds the padded coefficient with the random boundary
(rbc_build_velocity), then for every shot rbc_fwi_forward (modeling, residual,
misfit) and keeps only the residual and the two last panels of the shot.
backward: for every shot rbc_fwi_backward rebuilds the source wavefield
backwards from those panels -- the random boundary makes the recursion
reversible, so nothing is stored or checkpointed -- while it runs the exact
discrete adjoint, and accumulates dJ/dv on the interior.  All arithmetic runs
in librbc's kernels; this module only sequences the calls.
"""
from __future__ import annotations

import torch

from . import _native as N


class FWIMisfit(torch.autograd.Function):
    @staticmethod
    def forward(fctx, v_int, grid, shots, wavelet, rec, dobs, rbc):
        """v_int: interior velocity (nz, nx) fp32 CUDA; shots: list of source
        nodes; dobs: list of (nrec, nt+1) records; rbc: (v_lo, v_hi, v_max, seed)."""
        dev = v_int.device
        a = torch.empty(grid.padded, dtype=torch.float32, device=dev)
        N.rbc_build_velocity(grid, v_int.detach().contiguous(), *rbc[:3], rbc[3], 0, None, a)
        ctx = N.rbc_create(grid, a)
        misfit = torch.zeros(1, dtype=torch.float64, device=dev)
        resids, panels = [], []
        try:
            for src, d in zip(shots, dobs):
                r = torch.empty_like(d)
                p = torch.empty((2,) + tuple(grid.padded), dtype=torch.float32, device=dev)
                N.rbc_fwi_forward(ctx, src, wavelet, rec, d, r, misfit, p)
                resids.append(r)
                panels.append(p)
        except Exception:
            N.rbc_destroy(ctx)
            raise
        if not fctx.needs_input_grad[0]:
            N.rbc_destroy(ctx)   # no backward will come
            ctx = None
        fctx.rbc_ctx = ctx
        fctx.grid, fctx.shots, fctx.rec = grid, shots, rec
        fctx.save_for_backward(wavelet, *resids, *panels)
        return misfit.to(torch.float32).reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        saved = fctx.saved_tensors
        wavelet = saved[0]
        n = len(fctx.shots)
        resids, panels = saved[1:1 + n], saved[1 + n:1 + 2 * n]
        grid = fctx.grid
        g = torch.zeros(grid.interior, dtype=torch.float32, device=wavelet.device)
        try:
            for src, r, p in zip(fctx.shots, resids, panels):
                N.rbc_fwi_backward(fctx.rbc_ctx, src, wavelet, fctx.rec, r, p, g)
        finally:
            N.rbc_destroy(fctx.rbc_ctx)
        return g * grad_out.to(g.dtype), None, None, None, None, None, None


def fwi_misfit(v_int, grid, shots, wavelet, rec, dobs, rbc):
    """J(v) = sum over shots of 1/2 ||record - dobs||^2, differentiable in v_int."""
    return FWIMisfit.apply(v_int, grid, shots, wavelet, rec, dobs, rbc)
