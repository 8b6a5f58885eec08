"""Shared drivers for the GPU parity tests: run one shot through the C ABI and
through the FP64 oracle on the same seeded inputs (the oracle gets the inputs
rounded to the ABI's fp32, and builds its own random boundary)."""
import numpy as np

import oracle
import workloads as W

TOL = 1e-4   # relative L2, GPU fp32 vs oracle fp64


def rel(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    ny = np.linalg.norm(y)
    return float(np.linalg.norm(x - y) / (ny if ny > 0 else 1.0))


ILLUM = 1e-4  # image compared where den >= ILLUM * max(den)


def rel_image(g_img, o_img, o_den):
    """Relative L2 of the image over the illuminated region.  Where the source
    wavefield never arrives (den below ILLUM of its maximum), the ratio
    num / (den + eps max den) only scales rounding noise of the fp32
    reconstruction by 1 / (eps max den); the integrals themselves are compared
    everywhere."""
    m = o_den >= ILLUM * o_den.max()
    return rel(np.asarray(g_img)[m], np.asarray(o_img)[m]), float(m.mean())


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def grid_of(R, w):
    return R.make_grid(w.ndim, w.nx, w.ny, w.nz, w.nb, w.h, w.dt, w.nt)


def gpu_build(R, torch, w, v, mode=0):
    g = grid_of(R, w)
    vt = torch.tensor(np.asarray(v, np.float32), device="cuda")
    a = torch.empty(g.padded, dtype=torch.float32, device="cuda")
    vp = torch.empty(g.padded, dtype=torch.float32, device="cuda")
    R.rbc_build_velocity(g, vt, w.v_lo, w.v_hi, w.v_max, w.rbc_seed, mode, vp, a)
    return g, a, vp


def oracle_a(w, v, mode=0):
    vp = oracle.rbc_velocity(f32(v), w.nb, w.v_lo, w.v_hi, w.v_max, w.rbc_seed, mode)
    a64, a32 = oracle.coef(vp, w.dt, w.h)
    return vp, a32


def gpu_shot(R, torch, w, v, src, rec, wav, seis_in=None, snaps=(), reinject=True, v_rtm=None):
    """Model (with v) and migrate (with v_rtm, default v) one shot on the GPU."""
    g, a, _ = gpu_build(R, torch, w, v)
    wt = torch.tensor(np.asarray(wav, np.float32), device="cuda")
    rec = np.asarray(rec, np.int32).reshape(-1, 3)
    nrec = rec.shape[0]
    seis = torch.zeros((nrec, w.nt + 1), dtype=torch.float32, device="cuda")
    out = {}
    ctx = R.rbc_create(g, a)
    try:
        if snaps:
            pf = torch.zeros((len(snaps),) + g.padded, dtype=torch.float32, device="cuda")
            R.rbc_set_snapshots(ctx, snaps, pf=pf)
        R.rbc_model(ctx, src, wt, rec, seis)
        if snaps:
            out["pf"] = pf.cpu().numpy()
            R.rbc_set_snapshots(ctx, [])
        prev = torch.zeros(g.padded, dtype=torch.float32, device="cuda")
        last = torch.zeros_like(prev)
        R.rbc_get_panels(ctx, prev, last)
        out["prev"], out["last"] = prev.cpu().numpy(), last.cpu().numpy()
    finally:
        R.rbc_destroy(ctx)
    out["seis"] = seis.cpu().numpy()
    if v_rtm is not None:
        g, a, _ = gpu_build(R, torch, w, v_rtm)
    ctx = R.rbc_create(g, a)
    try:
        d = seis if seis_in is None else torch.tensor(np.asarray(seis_in, np.float32), device="cuda")
        num = torch.zeros(g.interior, dtype=torch.float32, device="cuda")
        den = torch.zeros_like(num)
        if snaps:
            pr = torch.zeros((len(snaps),) + g.padded, dtype=torch.float32, device="cuda")
            pb = torch.zeros_like(pr)
            R.rbc_set_snapshots(ctx, snaps, pr=pr, pb=pb)
        R.rbc_rtm_shot(ctx, src, wt, rec, d, R.RBC_REINJECT_SOURCE if reinject else 0, num, den)
        img = torch.zeros_like(num)
        R.rbc_image_stack(g, num, den, 1e-6, 0, 0, g, img)
        torch.cuda.synchronize()
        out.update(num=num.cpu().numpy(), den=den.cpu().numpy(), img=img.cpu().numpy())
        if snaps:
            out["pr"], out["pb"] = pr.cpu().numpy(), pb.cpu().numpy()
    finally:
        R.rbc_destroy(ctx)
    return out


def oracle_shot(w, v, src, rec, wav, seis_in=None, snaps=(), reinject=True, v_rtm=None):
    _, a32 = oracle_a(w, v)
    a = a32.astype(np.float64)
    wav = f32(wav)
    rec = np.asarray(rec, np.int32).reshape(-1, 3)
    m = oracle.model(a, w.h, w.nt, src, wav, rec, snaps=snaps)
    out = dict(seis=m["seis"], prev=m["p_prev"], last=m["p_last"], pf=m["snaps"])
    if v_rtm is not None:
        a = oracle_a(w, v_rtm)[1].astype(np.float64)
    d = m["seis"] if seis_in is None else f32(seis_in)
    r = oracle.rtm_shot(a, w.h, w.nt, src, wav, rec, d, w.nb,
                        (w.nx, w.ny if w.ndim == 3 else 1, w.nz), reinject=reinject, snaps=snaps)
    out.update(num=r["num"], den=r["den"], img=oracle.image(r["num"], r["den"], 1e-6),
               pr=r["pr"], pb=r["pb"])
    return out


def case_2d(name, nx, nz, nb, nt, seed=0, src=None, rec=None, layered=True):
    w = W.scaled(W.SMALL_2D, nx=nx, nz=nz, nb=nb, nt=nt, name=name)
    w = W.dataclasses.replace(w, rbc_seed=seed + 1)
    if layered:
        v = W.three_layers(nx, nz, (max(1, nz // 3), max(2, 2 * nz // 3)))
    else:
        v = np.random.default_rng(seed).uniform(1500, 3500, (nz, nx))
    src = W.source_at(w, nx // 2, depth=min(1, nz - 1)) if src is None else np.asarray(src, np.int32)
    rec = W.surface_line(w, depth=min(1, nz - 1)) if rec is None else np.asarray(rec, np.int32)
    return w, v, src, rec, W.ricker(nt, w.dt, w.f_peak)


def case_3d(name, nx, ny, nz, nb, nt, seed=0):
    w = W.scaled(W.SHOT_3D, nx=nx, ny=ny, nz=nz, nb=nb, nt=nt, name=name)
    w = W.dataclasses.replace(w, rbc_seed=seed + 3)
    v = W.dipping_salt_3d(nx, ny, nz, seed + 5)
    src = W.source_at(w, nx // 2, ny // 2, depth=1)
    rec = W.surface_grid(w, depth=1, step=3)
    return w, v, src, rec, W.ricker(nt, w.dt, w.f_peak)
