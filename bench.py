#!/usr/bin/env python
"""Benchmark of the RTM-with-random-boundaries hot path on GB300.

Workload (default): the 2-D survey -- 240 shots on a 2301 x 751 interior grid
at 4 m (plus a 60-cell random boundary: 2421 x 871 padded nodes), seeded
faulted-layered true model 1500-5500 m/s, migration model = Gaussian-smoothed
slowness, 25 Hz Ricker, dt 0.4 ms x 12500 steps (5 s), 460 fixed-spread
receivers every 5 cells at depth 1, image stacked over shots.

One STEP = Algorithm 3 (RTM with wavefield reconstruction) for a batch of
shots: forward modeling with source injection, the fused reverse pass
(reconstruction of the source wavefield, receiver back-propagation with
injection, both integrals of the imaging condition), then the image ratio and
the stack.  The observed records are modeled beforehand in the true model
(untimed setup: the step's input data, resident in HBM).  With the default
--steps 30 and 8 shots per step the timed region migrates the whole survey.

`value` is grid-point updates per second (3 wave equations per step, the
paper's count), device-timed with CUDA events, L2 flushed between steps.
`e2e` repeats the timed loop through host buffers: every step copies its
records from pinned host memory and reads the stacked image back.

--impl reference times the FP64 CPU oracle (the only reference this repo
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gpts/s stencil updates & s per RTM shot vs HBM roofline; learned vs K-stack"
EPS_REL = 1e-6
L2_FLUSH_BYTES = 256 << 20
ORACLE_SAMPLE_STEPS = 200     # cpu_baseline: one full-grid shot with this many time steps
REFERENCE_STEP_STEPS = 40     # --impl reference: per step, one full-grid shot of this many steps


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="default 30 (survey2d), 3 (shot3d)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--shots-per-step", type=int, default=None, help="default 8 (survey2d), 1 (shot3d)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-3d", action="store_true",
                   help="survey2d: skip the 3-D shot sub-record (one 500 x 500 x 300 + 40 shot of 3000 steps "
                        "after the survey; also skipped with --nt / --interior and on more than one GPU)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--nt", type=int, default=None,
                   help="record length override (default: the workload's full record); only for "
                        "small profiler captures")
    p.add_argument("--interior", type=int, nargs="+", default=None,
                   help="interior size override (nx nz | nx ny nz); only for small profiler captures")
    p.add_argument("--method", choices=["rbc", "storage"], default="rbc",
                   help="survey2d / shot3d: rbc = Algorithm 3 (reconstruction through the random boundary, "
                        "default); storage = Algorithm 2 with the source wavefield kept in device memory every "
                        "k steps, k from Eq. 7 with f_max = 2.5 x the peak frequency")
    p.add_argument("--denoise-models", type=int, default=512, help="denoise: training models")
    p.add_argument("--denoise-size", type=int, default=96, help="denoise: training image size")
    p.add_argument("--denoise-steps", type=int, default=20000, help="denoise: Adam steps (batch 32)")
    p.add_argument("--denoise-nb", type=int, default=None, help="denoise: boundary cells (default size / 4)")
    p.add_argument("--denoise-nt", type=int, default=None, help="denoise: time steps (default 6.5 x size)")
    p.add_argument("--denoise-shots", type=int, default=4, help="denoise: shots per model")
    p.add_argument("--cnn-batch", type=int, nargs=3, default=[32, 512, 512],
                   help="cnn: images, height, width of one training / inference batch")
    p.add_argument("--workload", choices=["survey2d", "shot3d", "batch2d", "denoise", "cnn", "fwi"], default="survey2d",
                   help="survey2d: the 240-shot 2-D survey (default); shot3d: one 3-D shot on "
                        "500 x 500 x 300 + 40 (one step = one RTM shot); batch2d: 64 shots of "
                        "400-1200 columns x 600 rows in one launch per time step (one step = the batch); "
                        "fwi: the FWI misfit and velocity gradient of 4 shots on 300 x 300 + 50 through "
                        "the autograd function (one step = one gradient)")
    a = p.parse_args()
    if a.steps is None:
        a.steps = {"survey2d": 30, "shot3d": 3, "batch2d": 5, "denoise": 3, "cnn": 20, "fwi": 20}[a.workload]
    if a.shots_per_step is None:
        a.shots_per_step = 8 if a.workload == "survey2d" else 1
    return a


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.dev = device_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.dev, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def smi_device_id(torch, dev_index: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        first = vis.split(",")[dev_index] if vis else str(dev_index)
        return first


# --------------------------------------------------------------- workload ---
def shot_plan(nshots_total: int, steps: int, warmup: int, per_step: int, rank: int, world: int):
    """Shots of every (warm-up then timed) step on this rank: disjoint across
    ranks within a step, cycling through the survey."""
    from paper_2204_03380_gb300.survey import shard_shots
    return shard_shots(nshots_total, rank, world, per_step, steps, warmup)


def updates_per_shot(w) -> int:
    # forward nt, reconstruction nt - 1, receiver wavefield nt updates per node
    return w.npad * (3 * w.nt - 1)


def storage_phase_bytes(w, stride):
    """Algorithmic bytes of Algorithm 2's two phases: nt leapfrog steps each
    (16 B per padded node) plus, at the kept levels, the interior store
    (read 4 + write 4) in the forward phase and the imaging read of the store,
    of pbar and the num/den read-modify-write (4 + 4 + 16) in the reverse."""
    nint = w.nx * (w.ny if w.ndim == 3 else 1) * w.nz
    kept = w.nt // stride + 1
    return 16 * w.npad * w.nt + 8 * nint * kept, 16 * w.npad * w.nt + 24 * nint * kept


def rev_bytes_per_launch(w) -> int:
    """Algorithmic bytes of one fused reverse launch: a (4) + p^R n, n+1->n-1
    (4 + 8) + pbar (4 + 8) per padded node, num/den read-modify-write (16) per
    interior node."""
    nint = w.nx * (w.ny if w.ndim == 3 else 1) * w.nz
    return 28 * w.npad + 16 * nint


def fwd_bytes_per_launch(w) -> int:
    return 16 * w.npad


def load_workload(W, args):
    """Workload preset, its inputs and one source node per shot (padded frame)."""
    if args.workload == "survey2d":
        w = W.SURVEY_2D
        if args.interior:
            w = W.scaled(w, nx=args.interior[0], nz=args.interior[-1], name=f"{w.name}_int{args.interior}")
        if args.nt:
            w = W.dataclasses.replace(w, nt=args.nt, name=f"{w.name}_nt{args.nt}")
        inp = W.survey_2d_inputs(w)
        inp["srcs"] = [W.source_at(w, int(x)) for x in inp["shots"]]
    else:
        w = W.SHOT_3D
        if args.interior:
            nx, ny, nz = args.interior
            w = W.scaled(w, nx=nx, ny=ny, nz=nz, name=f"3d_{nx}x{ny}x{nz}_nb{w.nb}")
        if args.nt:
            w = W.dataclasses.replace(w, nt=args.nt, name=f"{w.name}_nt{args.nt}")
        inp = W.shot_3d_inputs(w)
        inp["v_true"] = inp["v"]
        inp["v_mig"] = W.smooth_slowness(inp["v"], 8.0)
        inp["srcs"] = [inp["src"]]
        inp["shots"] = np.array([w.nx // 2])
    return w, inp


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the stencil
# kernels from ncu captures (profiles/), recorded with a hash of the kernel
# sources they were taken on: a capture of older sources reads as null.
#   k_rev2d_tile on the 2-D survey grid, warm L2 as in the time loop (one-pass
#   metrics capture, mean of three launches): the shot's fields stay in L2.
#   3-D kernels: captured on the 380 x 380 x 280 grid as a multiple of their
#   algorithmic bytes; the traffic of their tiles grows in proportion to the
#   nodes, so a full 580 x 580 x 380 launch gets that multiple of its own.
_SRC2 = ["rbc_kernels.cu", "rbc_tile2d.cuh", "rbc_stencil.cuh", "rbc_internal.cuh"]
_SRC3 = ["rbc_kernels3d.cu", "rbc_stencil.cuh", "rbc_internal.cuh"]
TRAFFIC = {
    "k_rev2d_tile": {"sources": _SRC2, "sha1": "f860ce948d6f75a4", "bytes_per_launch": 1.02e6, "ratio": None},
    "k_rev3d_tma": {"sources": _SRC3, "sha1": "b0ea2b88596cbbf5", "bytes_per_launch": None, "ratio": 1.122},
    "k_fwd3d_tma": {"sources": _SRC3, "sha1": "b0ea2b88596cbbf5", "bytes_per_launch": None, "ratio": 1.087},
}


def sources_sha(files):
    import hashlib
    m = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2204_03380_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return m.hexdigest()[:16]


def kernel_traffic(kernel, algorithmic_bytes):
    """Per-launch DRAM traffic of a kernel from its recorded ncu capture, or
    None when the kernel sources changed since."""
    t = TRAFFIC[kernel]
    if sources_sha(t["sources"]) != t["sha1"]:
        return None
    return t["bytes_per_launch"] if t["bytes_per_launch"] else t["ratio"] * algorithmic_bytes


def reverse_traffic(ndim, algorithmic_bytes):
    return kernel_traffic("k_rev2d_tile" if ndim == 2 else "k_rev3d_tma", algorithmic_bytes)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ----------------------------------------------------------------- oracle ---
def oracle_rtm_sample(w, inp, nsteps: int):
    """Time the FP64 oracle (as it stands) on one full-grid shot of `nsteps`."""
    import oracle
    import workloads as W
    ws = W.dataclasses.replace(w, nt=nsteps)
    vp = oracle.rbc_velocity(inp["v_mig"].astype(np.float32), ws.nb, ws.v_lo, ws.v_hi, ws.v_max, ws.rbc_seed)
    a = oracle.coef(vp, ws.dt, ws.h)[1].astype(np.float64)
    src = inp["srcs"][0]
    rec = inp["rec"]
    wav = inp["wavelet"][:nsteps]
    seis = np.zeros((len(rec), nsteps + 1))
    t0 = time.perf_counter()
    r = oracle.rtm_shot(a, ws.h, nsteps, src, wav, rec, seis, ws.nb,
                        (ws.nx, ws.ny if ws.ndim == 3 else 1, ws.nz))
    img = oracle.image(r["num"], r["den"], EPS_REL)
    dt = time.perf_counter() - t0
    assert np.isfinite(img).all()
    return updates_per_shot(ws) / dt / 1e9, dt


def oracle_cnn_sample(H, W, backward=False):
    """Time the FP64 oracle network (as it stands) on one H x W image:
    forward, or forward + backward.  Returns seconds."""
    import oracle.cnn as OC
    params = OC.init_params(0)
    x = np.random.default_rng(0).standard_normal((1, H, W))
    t0 = time.perf_counter()
    y, cache = OC.forward(params, x)
    if backward:
        OC.backward(params, cache, y - x)
    return time.perf_counter() - t0


def cores_used():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n and n.isdigit() else (os.cpu_count() or 1)


def run_batch(args, rank, world):
    """batch2d: one step = rbc_batch_rtm over the 64 uneven-aperture shots."""
    import torch
    import paper_2204_03380_gb300 as R
    import workloads as W
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = W.BATCH_2D
    if args.nt:
        w = W.dataclasses.replace(w, nt=args.nt, name=f"{w.name}_nt{args.nt}")
    inp = W.batch_2d_inputs(w)
    dev = torch.device("cuda", local)
    wav = torch.tensor(inp["wavelet"], dtype=torch.float32, device=dev)
    a_mig, seis = [], []
    for sh in inp["shots"]:
        g = R.make_grid(2, sh["width"], 1, w.nz, w.nb, w.h, w.dt, w.nt)
        pair = []
        for v in (inp["v_true"], inp["v_mig"]):
            vw = torch.tensor(np.ascontiguousarray(v[:, sh["off_x"]:sh["off_x"] + sh["width"]]),
                              dtype=torch.float32, device=dev)
            a = torch.empty(g.padded, dtype=torch.float32, device=dev)
            R.rbc_build_velocity(g, vw, w.v_lo, w.v_hi, w.v_max, w.rbc_seed, 0, None, a)
            pair.append(a)
        ctx = R.rbc_create(g, pair[0])
        d = torch.empty((len(sh["rec"]), w.nt + 1), dtype=torch.float32, device=dev)
        R.rbc_model(ctx, sh["src"], wav, sh["rec"], d)
        torch.cuda.synchronize()
        R.rbc_destroy(ctx)
        a_mig.append(pair[1])
        seis.append(d)
    base = R.make_grid(2, 1, 1, w.nz, w.nb, w.h, w.dt, w.nt)
    b = R.rbc_batch_create(base, [sh["width"] for sh in inp["shots"]], a_mig)
    info = R.rbc_batch_info(b)
    image = torch.zeros((w.nz, w.nx), dtype=torch.float32, device=dev)
    shots = [dict(src=sh["src"], rec=sh["rec"], seis=d, off_x=sh["off_x"]) for sh, d in zip(inp["shots"], seis)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        R.rbc_batch_rtm(b, shots, wav, R.RBC_REINJECT_SOURCE, EPS_REL, image)
    barrier()
    smi = ClockSampler(smi_device_id(torch, local))
    smi.start()
    time.sleep(0.3)
    R.rbc_launch_count(reset=True)
    R.rbc_batch_timing(b, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record()
    for _ in range(args.steps):
        flush.zero_()
        R.rbc_batch_rtm(b, shots, wav, R.RBC_REINJECT_SOURCE, EPS_REL, image)
    ev1.record()
    barrier()
    phases = R.rbc_batch_timing(b, False)
    launches = R.rbc_launch_count()
    clocks = smi.stop()
    el = ev0.elapsed_time(ev1) / 1e3
    if dist is not None:
        t = torch.tensor([el], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    npads = [(sh["width"] + 2 * w.nb) * (w.nz + 2 * w.nb) for sh in inp["shots"]]
    nints = [sh["width"] * w.nz for sh in inp["shots"]]
    upd = sum(npads) * (3 * w.nt - 1) * args.steps * world
    value = upd / el / 1e9
    e2e = None
    if not args.no_e2e:
        host = [d.cpu().pin_memory() for d in seis]
        stage = [torch.empty_like(d) for d in seis]
        img_host = torch.empty(image.shape, dtype=torch.float32).pin_memory()
        shots_s = [dict(sh, seis=st) for sh, st in zip(shots, stage)]
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            for st, hs in zip(stage, host):
                st.copy_(hs, non_blocking=True)
            R.rbc_batch_rtm(b, shots_s, wav, R.RBC_REINJECT_SOURCE, EPS_REL, image)
            img_host.copy_(image, non_blocking=True)
        barrier()
        el_e = time.perf_counter() - t0
        e2e = {"value": upd / world / el_e / 1e9 * world, "unit": "Gpts/s",
               "h2d_bytes_per_step": int(sum(d.numel() for d in seis)) * 4,
               "d2h_bytes_per_step": int(image.numel()) * 4}
    R.rbc_batch_destroy(b)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    rev_bytes = sum(28 * p + 16 * q for p, q in zip(npads, nints))
    rev_s = phases["rev_ms"] / 1e3 / max(phases["rev_launches"], 1)
    fwd_s = phases["fwd_ms"] / 1e3 / max(phases["fwd_launches"], 1)
    achieved = rev_bytes / rev_s / 1e9
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle's RTM of shot 0 (its own window and record) over the first
        # nsamp steps, about 6e9 stencil updates
        import oracle
        sh = inp["shots"][0]
        ws = W.dataclasses.replace(w, nx=sh["width"])
        nsamp = int(max(10, min(w.nt, 6e9 / (3 * npads[0]))))
        vw = np.ascontiguousarray(inp["v_mig"][:, sh["off_x"]:sh["off_x"] + sh["width"]]).astype(np.float32)
        ao = oracle.coef(oracle.rbc_velocity(vw, w.nb, w.v_lo, w.v_hi, w.v_max, w.rbc_seed), w.dt, w.h)[1]
        d0 = seis[0].cpu().numpy()[:, :nsamp + 1].astype(np.float64)
        t0 = time.perf_counter()
        r = oracle.rtm_shot(ao.astype(np.float64), w.h, nsamp, sh["src"], inp["wavelet"][:nsamp], sh["rec"], d0,
                            w.nb, (ws.nx, 1, w.nz))
        dt_o = time.perf_counter() - t0
        assert np.isfinite(r["num"]).all()
        cpu = {"value": npads[0] * (3 * nsamp - 1) / dt_o / 1e9, "unit": "Gpts/s", "cores": cores_used(),
               "kind": "oracle", "sample": f"oracle RTM of shot 0 ({sh['width']} + {2 * w.nb} columns), "
                                           f"{nsamp} of the {w.nt} steps: {dt_o:.1f} s"}
    out = {"metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "shots": len(shots), "widths": [min(s["width"] for s in inp["shots"]),
                                                                         max(s["width"] for s in inp["shots"])],
                      "nt": w.nt, "autotuned": info, "s_per_shot": el / args.steps / len(shots),
                      "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
           "roofline": {"bound": "hbm", "kernel": "k_rev2d_batch (fused reverse pass, all shots)",
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s",
                        "traffic": None, "bytes_per_launch": rev_bytes, "launch_us": rev_s * 1e6,
                        "forward_kernel": {"kernel": "k_fwd2d_batch", "launch_us": fwd_s * 1e6,
                                           "achieved": 16 * sum(npads) / fwd_s / 1e9}},
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_denoise(args, rank, world):
    """denoise: the learned stand-in for the 16-realization stack.

    Quality: a training set of single-realization / 16-stack image pairs is
    migrated by the batched path from seeded faulted-layered models, the CNN is
    trained by librbc's kernels, and its error to the 16-stack is measured on
    held-out models.  Speed: one 3-D RTM of the 800 x 800 x 400 image (+40
    boundary) is timed; the 16-stack costs 16 such migrations; the network
    denoises the volume x-z slice by slice.  value = 16-stack time / network
    time (one step = one slice-wise pass over the volume)."""
    import torch
    import paper_2204_03380_gb300 as R
    from paper_2204_03380_gb300 import denoise as D
    import workloads as W
    if rank != 0:
        return
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = args.denoise_size
    K, S = 16, args.denoise_shots
    nb_d = args.denoise_nb or n // 4
    nt_d = args.denoise_nt or int(6.5 * n)

    def image_set(M, seed):
        w = W.scaled(W.SMALL_2D, nx=n, nz=n, nb=nb_d, nt=nt_d, name="dn")
        vt = [W.faulted_layers(n, n, seed + m, 1500.0, 4000.0, nlayers=8, nfaults=2) for m in range(M)]
        vm = [W.smooth_slowness(v, 4.0) for v in vt]
        g = R.make_grid(2, n, 1, n, w.nb, w.h, w.dt, w.nt)
        shots = [W.source_at(w, int(x)) for x in np.linspace(n / (2 * S), n - n / (2 * S), S).astype(int)]
        return D.rtm_realizations(R, g, vt, vm, K, shots, W.surface_line(w), W.ricker(w.nt, w.dt, w.f_peak),
                                  (1500.0, 4000.0, 4000.0))

    t0 = time.perf_counter()
    train, held = image_set(args.denoise_models, 0), image_set(16, 100000)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    x, t, _ = D.normalized_pairs(train)
    x, t = torch.cat([x, x.flip(-1)]), torch.cat([t, t.flip(-1)])
    net = D.Denoiser(seed=1)
    t0 = time.perf_counter()
    ns = args.denoise_steps
    for lr, st, sd in ((2e-3, ns // 2, 0), (5e-4, ns // 4, 1), (1e-4, ns // 4, 2)):
        net.fit(x, t, steps=st, batch=32, lr=lr, seed=sd)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    xs, ts, _ = D.normalized_pairs(held)
    e_single, e_net = D.rel_l2(xs, ts), D.rel_l2(net(xs), ts)
    e_half = D.rel_l2(held.images[:, :8].mean(1) / D.normalized_pairs(held)[2], ts)

    # 3-D: one RTM of the 800 x 800 x 400 image (realization 0)
    w3 = W.scaled(W.SHOT_3D, nx=800, ny=800, nz=400, nb=40, name="3d_800x800x400_nb40_3000steps")
    if args.nt:
        w3 = W.dataclasses.replace(w3, nt=args.nt)
    inp = W.shot_3d_inputs(w3)
    g3 = R.make_grid(3, w3.nx, w3.ny, w3.nz, w3.nb, w3.h, w3.dt, w3.nt)
    wav = torch.tensor(inp["wavelet"], dtype=torch.float32, device=dev)
    rec = W.surface_grid(w3, step=4)
    a = torch.empty(g3.padded, dtype=torch.float32, device=dev)
    R.rbc_build_velocity(g3, torch.tensor(inp["v"], dtype=torch.float32, device=dev), w3.v_lo, w3.v_hi,
                         w3.v_max, w3.rbc_seed, 0, None, a)
    ctx = R.rbc_create(g3, a)
    seis = torch.empty((len(rec), w3.nt + 1), dtype=torch.float32, device=dev)
    R.rbc_model(ctx, inp["src"], wav, rec, seis)
    R.rbc_destroy(ctx)
    R.rbc_build_velocity(g3, torch.tensor(W.smooth_slowness(inp["v"], 8.0), dtype=torch.float32, device=dev),
                         w3.v_lo, w3.v_hi, w3.v_max, w3.rbc_seed, 0, None, a)
    ctx = R.rbc_create(g3, a)
    del a
    num = torch.zeros(g3.interior, dtype=torch.float32, device=dev)
    den = torch.zeros_like(num)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    R.rbc_rtm_shot(ctx, inp["src"], wav, rec, seis, R.RBC_REINJECT_SOURCE, num, den)
    img = torch.zeros_like(num)
    R.rbc_image_stack(g3, num, den, EPS_REL, 0, 0, g3, img)
    ev1.record()
    torch.cuda.synchronize()
    t_rtm = ev0.elapsed_time(ev1) / 1e3
    R.rbc_destroy(ctx)
    del num, den, seis
    vol = img / img.pow(2).mean().sqrt()
    del img
    for _ in range(args.warmup):
        net.denoise_volume(vol)
    torch.cuda.synchronize()
    smi = ClockSampler(smi_device_id(torch, 0))
    smi.start()
    time.sleep(0.3)
    R.rbc_launch_count(reset=True)
    ev0.record()
    for _ in range(args.steps):
        out = net.denoise_volume(vol)
    ev1.record()
    torch.cuda.synchronize()
    launches = R.rbc_launch_count()
    clocks = smi.stop()
    t_inf = ev0.elapsed_time(ev1) / 1e3 / args.steps
    assert torch.isfinite(out).all()
    px = w3.nx * w3.ny * w3.nz
    flops = 56448.0 * px
    peaks = measured_peaks()
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    achieved = flops / t_inf / 1e12
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle network on one x-z slice, scaled to the volume's slices
        dt_o = oracle_cnn_sample(w3.nz, w3.nx)
        cpu = {"value": dt_o * w3.ny, "unit": "s per volume (oracle network, extrapolated)",
               "cores": cores_used(), "kind": "oracle",
               "sample": f"oracle.cnn forward of 1 of the {w3.ny} x-z slices ({w3.nz}x{w3.nx}): {dt_o:.1f} s"}
    out = {"metric": METRIC, "value": 16 * t_rtm / t_inf, "unit": "x (16-realization 3-D stack time / network time)",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_inf * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
           "data": "synthetic",
           "config": {"workload": "denoise: train " + f"{args.denoise_models} pairs of {n}x{n} (K=16, {S} shots, "
                                  + f"nb {nb_d}, {nt_d} steps); "
                                  + f"infer {w3.ny} x-z slices of {w3.nz}x{w3.nx}",
                      "heldout_rel_l2_to_16stack": {"single_realization": e_single, "network": e_net,
                                                     "8_stack": e_half, "target": 5e-2},
                      "train_data_s": t_data, "train_s": t_train, "rtm_3d_s": t_rtm, "stack16_s": 16 * t_rtm,
                      "inference_s": t_inf},
           "roofline": {"bound": "tensor", "kernel": "k_conv_tc (tcgen05: layers 1-2 fused, layers 3-4, and the 32 -> 1 layer 5)", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "peak_source": "measured bf16 (MEASURED_PEAKS.json bf16_tflops)", "traffic": None},
           "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_cnn(args, rank, world):
    """cnn: the denoiser's kernels on their own.  One step = one training step
    (forward, MSE, backward, Adam) on a batch of seeded random images; the
    inference forward of the same batch is timed separately and gives the
    tensor-core roofline line (56 448 flop per pixel over the 5 layers)."""
    import torch
    from paper_2204_03380_gb300 import denoise as D
    if rank != 0:
        return
    torch.cuda.set_device(0)
    n, H, Wd = args.cnn_batch
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((n, H, Wd), generator=g, device="cuda")
    t = torch.randn((n, H, Wd), generator=g, device="cuda")
    net = D.Denoiser(seed=1)
    import paper_2204_03380_gb300 as R
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        net.train_step(x, t, 1e-5)
    torch.cuda.synchronize()
    smi = ClockSampler(smi_device_id(torch, 0))
    smi.start()
    time.sleep(0.3)
    R.rbc_launch_count(reset=True)
    ev0.record()
    for _ in range(args.steps):
        net.train_step(x, t, 1e-5)
    ev1.record()
    torch.cuda.synchronize()
    launches = R.rbc_launch_count()
    clocks = smi.stop()
    t_train = ev0.elapsed_time(ev1) / 1e3 / args.steps
    # end to end: the batch from pinned host memory every step, the loss read back
    e2e = None
    if not args.no_e2e:
        xh, th = x.cpu().pin_memory(), t.cpu().pin_memory()
        xs, ts = torch.empty_like(x), torch.empty_like(t)
        loss_h = torch.empty((1,), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            xs.copy_(xh, non_blocking=True)
            ts.copy_(th, non_blocking=True)
            loss_h.copy_(net.train_step(xs, ts, 1e-5), non_blocking=True)
        torch.cuda.synchronize()
        el_e = time.perf_counter() - t0
        e2e = {"value": n * H * Wd * args.steps / el_e / 1e9, "unit": "Gpx/s (training: forward + backward + Adam)",
               "h2d_bytes_per_step": 2 * n * H * Wd * 4, "d2h_bytes_per_step": 8}
    cpu = None
    if not args.no_cpu_baseline:
        dt_o = oracle_cnn_sample(H, Wd, backward=True)
        cpu = {"value": H * Wd / dt_o / 1e9, "unit": "Gpx/s (forward + backward)", "cores": cores_used(),
               "kind": "oracle", "sample": f"oracle.cnn forward + backward of 1 image of {H}x{Wd}: {dt_o:.1f} s"}
    for _ in range(args.warmup):
        y = net(x)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        y = net(x)
    ev1.record()
    torch.cuda.synchronize()
    t_inf = ev0.elapsed_time(ev1) / 1e3 / args.steps
    assert torch.isfinite(y).all()
    px = n * H * Wd
    peaks = measured_peaks()
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    achieved = 56448.0 * px / t_inf / 1e12
    out = {"metric": METRIC, "value": px / t_train / 1e9, "unit": "Gpx/s (training: forward + backward + Adam)",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_train * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
           "data": "synthetic", "config": {"workload": f"cnn: batch of {n} images of {H}x{Wd}",
                                           "train_step_ms": t_train * 1e3, "inference_ms": t_inf * 1e3,
                                           "training_tflops": 3 * 56448.0 * px / t_train / 1e12,
                                           "l2": "working set larger than L2 (bf16 activations of 64 B per pixel "
                                                 "and layer)"},
           "roofline": {"bound": "tensor", "kernel": "k_conv_tc (tcgen05: layers 1-2 fused, layers 3-4, and the 32 -> 1 layer 5)", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "peak_source": "measured bf16 (MEASURED_PEAKS.json bf16_tflops)", "traffic": None},
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_fwi(args, rank, world):
    """fwi: one step = J(v) and dJ/dv for the 4-shot 300 x 300 model through
    the autograd function (rbc_fwi_forward per shot, then rbc_fwi_backward:
    reconstruction through the random boundary fused with the exact adjoint).
    Stencil updates per gradient: 3 nt - 1 per padded node per shot, as RTM."""
    import torch
    import paper_2204_03380_gb300 as R
    from paper_2204_03380_gb300.fwi import fwi_misfit, shot_streams
    import workloads as W
    if rank != 0:
        return
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = W.FWI_2D
    if args.nt:
        w = W.dataclasses.replace(w, nt=args.nt, name=f"{w.name}_nt{args.nt}")
    inp = W.fwi_2d_inputs(w)
    g = R.make_grid(2, w.nx, 1, w.nz, w.nb, w.h, w.dt, w.nt)
    wav = torch.tensor(inp["wavelet"], device=dev)
    rec, srcs = inp["rec"], inp["srcs"]
    rbc = (w.v_lo, w.v_hi, w.v_max, w.rbc_seed)
    # observed records from the true model (setup, untimed)
    a = torch.empty(g.padded, dtype=torch.float32, device=dev)
    R.rbc_build_velocity(g, torch.tensor(inp["v_true"], device=dev), *rbc[:3], rbc[3], 0, None, a)
    ctx = R.rbc_create(g, a)
    dobs = []
    for s in srcs:
        d = torch.empty((len(rec), w.nt + 1), dtype=torch.float32, device=dev)
        R.rbc_model(ctx, s, wav, rec, d)
        dobs.append(d)
    torch.cuda.synchronize()
    R.rbc_destroy(ctx)
    del a
    v0 = torch.tensor(inp["v0"], device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def gradient(obs, ev=None):
        v = v0.clone().requires_grad_(True)
        if ev:
            ev[0].record()
        J = fwi_misfit(v, g, srcs, wav, rec, obs, rbc)
        if ev:
            ev[1].record()
        J.backward()
        if ev:
            ev[2].record()
        return J, v.grad

    for _ in range(args.warmup):
        gradient(dobs)
    torch.cuda.synchronize()
    smi = ClockSampler(smi_device_id(torch, 0))
    smi.start()
    time.sleep(0.3)
    R.rbc_launch_count(reset=True)
    # per step: forward phase (all shots, modeling + residual) and backward
    # phase (all shots, reconstruction + adjoint + gradient), on the stream the
    # autograd function joins its shot streams to
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for k in range(args.steps):
        flush.zero_()
        J, grad = gradient(dobs, evs[k])
    ev1.record()
    torch.cuda.synchronize()
    launches = R.rbc_launch_count()
    clocks = smi.stop()
    el = ev0.elapsed_time(ev1) / 1e3
    t_f = sum(e[0].elapsed_time(e[1]) for e in evs) / 1e3 / args.steps
    t_b = sum(e[1].elapsed_time(e[2]) for e in evs) / 1e3 / args.steps
    t_grad = t_f + t_b
    upd = updates_per_shot(w) * len(srcs)
    value = upd * args.steps / el / 1e9
    nint = w.nx * w.nz
    rev_bytes = 28 * w.npad + 8 * nint        # gradient mode: num += pbar x increment
    # shots run concurrently (one stream each): launch time = phase time per
    # launch of one shot's loop, i.e. the launches of all shots share the phase
    rev_launch_s = t_b / (len(srcs) * (w.nt + 1))
    fwd_launch_s = t_f / (len(srcs) * w.nt)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = rev_bytes / rev_launch_s / 1e9
    # end to end: observed records from pinned host memory, gradient and misfit read back
    e2e = None
    if not args.no_e2e:
        host = [d.cpu().pin_memory() for d in dobs]
        stage = [torch.empty_like(d) for d in dobs]
        g_host = torch.empty((w.nz, w.nx), dtype=torch.float32).pin_memory()
        j_host = torch.empty((), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            for st, hs in zip(stage, host):
                st.copy_(hs, non_blocking=True)
            J, grad = gradient(stage)
            g_host.copy_(grad, non_blocking=True)
            j_host.copy_(J.detach(), non_blocking=True)
        torch.cuda.synchronize()
        el_e = time.perf_counter() - t0
        e2e = {"value": upd * args.steps / el_e / 1e9, "unit": "Gpts/s",
               "h2d_bytes_per_step": int(sum(d.numel() for d in dobs)) * 4,
               "d2h_bytes_per_step": int(w.nx * w.nz + 1) * 4}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        vp = oracle.rbc_velocity(inp["v0"], w.nb, w.v_lo, w.v_hi, w.v_max, w.rbc_seed)
        ao = oracle.coef(vp, w.dt, w.h)[1].astype(np.float64)
        t0 = time.perf_counter()
        oracle.fwi_grad(ao, w.h, w.dt, w.nt, srcs[0], inp["wavelet"], rec, dobs[0].cpu().numpy().astype(np.float64),
                        w.nb, (w.nx, 1, w.nz))
        dt_o = time.perf_counter() - t0
        cpu = {"value": updates_per_shot(w) / dt_o / 1e9, "unit": "Gpts/s", "cores": cores_used(), "kind": "oracle",
               "sample": f"oracle.fwi_grad of shot 0 (of {len(srcs)}), full {w.nt} steps: {dt_o:.2f} s"}
    out = {"metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "shots": len(srcs), "receivers": int(len(rec)), "nt": w.nt,
                      "s_per_gradient": t_grad, "forward_phase_s": t_f, "backward_phase_s": t_b,
                      "shot_streams": shot_streams(g, len(srcs)), "misfit": float(J.detach()),
                      "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
           "roofline": {"bound": "hbm", "kernel": "k_rev2d_tile<2, 4, 7, true> (reconstruction + exact adjoint + gradient; "
                                                  "shots on concurrent streams: backward phase / launches)",
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
                        "traffic": None, "bytes_per_launch": rev_bytes, "launch_us": rev_launch_s * 1e6,
                        "forward_kernel": {"kernel": "k_fwd2d", "launch_us": fwd_launch_s * 1e6,
                                           "achieved": 16 * w.npad / fwd_launch_s / 1e9}},
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out), flush=True)


def shot3d_subrecord(R, W, torch, dev, peaks, warmup=1, shots=1):
    """The 3-D shot workload (500 x 500 x 300 + 40 = 580 x 580 x 380 padded,
    3000 steps of 1 ms, 62 500 surface receivers): `shots` RTM shots of
    Algorithm 3 timed with CUDA events after `warmup` shots, on inputs
    resident in HBM (the 4 GB of fields exceed L2 by 30x).  Returns s per
    shot, Gpts/s, the HBM roofline of its two stencil kernels and the clocks
    sampled while it ran."""
    a3 = argparse.Namespace(workload="shot3d", interior=None, nt=None)
    w, inp = load_workload(W, a3)
    g = R.make_grid(3, w.nx, w.ny, w.nz, w.nb, w.h, w.dt, w.nt)
    a = torch.empty(g.padded, dtype=torch.float32, device=dev)
    R.rbc_build_velocity(g, torch.tensor(inp["v_true"], dtype=torch.float32, device=dev), w.v_lo, w.v_hi,
                         w.v_max, w.rbc_seed, 0, None, a)
    wav = torch.tensor(inp["wavelet"], dtype=torch.float32, device=dev)
    rec, src = inp["rec"], inp["srcs"][0]
    seis = torch.empty((len(rec), w.nt + 1), dtype=torch.float32, device=dev)
    ctx = R.rbc_create(g, a)
    R.rbc_model(ctx, src, wav, rec, seis)          # the shot's observed record (setup, untimed)
    torch.cuda.synchronize()
    R.rbc_destroy(ctx)
    R.rbc_build_velocity(g, torch.tensor(inp["v_mig"], dtype=torch.float32, device=dev), w.v_lo, w.v_hi,
                         w.v_max, w.rbc_seed, 0, None, a)
    ctx = R.rbc_create(g, a)
    del a
    num = torch.empty(g.interior, dtype=torch.float32, device=dev)
    den = torch.empty_like(num)
    image = torch.zeros_like(num)
    flags = R.RBC_REINJECT_SOURCE | R.RBC_ZERO_FIRST
    try:
        for _ in range(warmup):
            R.rbc_rtm_shot(ctx, src, wav, rec, seis, flags, num, den)
            R.rbc_image_stack(g, num, den, EPS_REL, 0, 0, g, image)
        torch.cuda.synchronize()
        smi = ClockSampler(smi_device_id(torch, dev.index or 0))
        smi.start()
        time.sleep(0.3)
        R.rbc_phase_timing(ctx, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(shots):
            R.rbc_rtm_shot(ctx, src, wav, rec, seis, flags, num, den)
            R.rbc_image_stack(g, num, den, EPS_REL, 0, 0, g, image)
        ev1.record()
        torch.cuda.synchronize()
        phases = R.rbc_phase_timing(ctx, False)
        clocks = smi.stop()
    finally:
        R.rbc_destroy(ctx)
    el = ev0.elapsed_time(ev1) / 1e3 / shots
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    rev_s = phases["rev_ms"] / 1e3 / max(phases["rev_launches"], 1)
    fwd_s = phases["fwd_ms"] / 1e3 / max(phases["fwd_launches"], 1)
    rb, fb = rev_bytes_per_launch(w), fwd_bytes_per_launch(w)
    src_note = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"
    return {"workload": w.name, "padded_grid": list(w.padded[::-1]), "nt": w.nt, "receivers": int(len(rec)),
            "shots_timed": shots, "s_per_shot": el, "value": updates_per_shot(w) / el / 1e9, "unit": "Gpts/s",
            "target_s_per_shot": 4.9,
            "roofline": {"bound": "hbm", "kernel": "k_rev3d_tma (fused reverse pass)",
                         "achieved": rb / rev_s / 1e9, "peak": peak, "unit": "GB/s", "frac": rb / rev_s / 1e9 / peak,
                         "peak_source": src_note, "traffic": kernel_traffic("k_rev3d_tma", rb),
                         "traffic_source": "ncu dram bytes of k_rev3d_tma on 380x380x280, scaled by the "
                                           "algorithmic bytes",
                         "bytes_per_launch": rb, "launch_us": rev_s * 1e6,
                         "forward_kernel": {"kernel": "k_fwd3d_tma", "achieved": fb / fwd_s / 1e9,
                                            "frac": fb / fwd_s / 1e9 / peak,
                                            "traffic": kernel_traffic("k_fwd3d_tma", fb),
                                            "launch_us": fwd_s * 1e6, "bytes_per_launch": fb}},
            "clocks": clocks}


def run_reference(args, rank, world):
    import workloads as W
    if rank != 0:
        return
    w, inp = load_workload(W, args)
    nsamp = REFERENCE_STEP_STEPS if w.ndim == 2 else 4
    for _ in range(args.warmup):
        oracle_rtm_sample(w, inp, nsamp)
    t0 = time.perf_counter()
    total_upd = 0
    for _ in range(args.steps):
        oracle_rtm_sample(w, inp, nsamp)
        total_upd += updates_per_shot(W.dataclasses.replace(w, nt=nsamp))
    el = time.perf_counter() - t0
    val = total_upd / el / 1e9
    sample = (f"per step one full-grid shot ({'x'.join(map(str, w.padded[::-1]))} padded) of Algorithm 3 "
              f"with {nsamp} of the {w.nt} time steps")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gpts/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": w.name, "reference": "FP64 CPU oracle (oracle/)"},
           "cpu_baseline": {"value": val, "unit": "Gpts/s", "cores": cores_used(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------- ours ---
def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch2d":
        run_batch(args, rank, world)
        return
    if args.workload == "denoise":
        run_denoise(args, rank, world)
        return
    if args.workload == "cnn":
        run_cnn(args, rank, world)
        return
    if args.workload == "fwi":
        run_fwi(args, rank, world)
        return
    import torch
    import paper_2204_03380_gb300 as R
    from paper_2204_03380_gb300.survey import reduce_image
    import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w, inp = load_workload(W, args)
    g = R.make_grid(w.ndim, w.nx, w.ny, w.nz, w.nb, w.h, w.dt, w.nt)
    dev = torch.device("cuda", local)
    a_true = torch.empty(g.padded, dtype=torch.float32, device=dev)
    a_mig = torch.empty_like(a_true)
    R.rbc_build_velocity(g, torch.tensor(inp["v_true"], dtype=torch.float32, device=dev), w.v_lo, w.v_hi,
                         w.v_max, w.rbc_seed, 0, None, a_true)
    R.rbc_build_velocity(g, torch.tensor(inp["v_mig"], dtype=torch.float32, device=dev), w.v_lo, w.v_hi,
                         w.v_max, w.rbc_seed, 0, None, a_mig)
    wav = torch.tensor(inp["wavelet"], dtype=torch.float32, device=dev)
    rec = inp["rec"]
    nrec = rec.shape[0]
    B = args.shots_per_step
    plan = shot_plan(w.nshots, args.steps, args.warmup, B, rank, world)
    needed = sorted({s for step in plan for s in step})
    srcs = {s: inp["srcs"][s] for s in needed}

    # observed records, modeled in the true model (setup, untimed)
    ctx_true = R.rbc_create(g, a_true)
    seis = {}
    for s in needed:
        d = torch.empty((nrec, w.nt + 1), dtype=torch.float32, device=dev)
        R.rbc_model(ctx_true, srcs[s], wav, rec, d)
        seis[s] = d
    torch.cuda.synchronize()
    R.rbc_destroy(ctx_true)

    ctx = R.rbc_create(g, a_mig)
    num = torch.empty(g.interior, dtype=torch.float32, device=dev)
    den = torch.empty_like(num)
    image = torch.zeros(g.interior, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flags = R.RBC_REINJECT_SOURCE | R.RBC_ZERO_FIRST

    storage = args.method == "storage"
    if storage:
        stride = R.rbc_nyquist_stride(w.dt, 2.5 * w.f_peak)
        store = torch.empty(R.rbc_storage_bytes(g, stride) // 4, dtype=torch.float32, device=dev)

    def migrate(shot, d):
        if storage:
            R.rbc_rtm_storage(ctx, srcs[shot], wav, rec, d, stride, store, R.RBC_ZERO_FIRST, num, den)
        else:
            R.rbc_rtm_shot(ctx, srcs[shot], wav, rec, d, flags, num, den)
        R.rbc_image_stack(g, num, den, EPS_REL, 0, 0, g, image)

    for s in range(args.warmup):
        for shot in plan[s]:
            migrate(shot, seis[shot])
    barrier()

    smi = ClockSampler(smi_device_id(torch, local))
    smi.start()
    time.sleep(0.3)
    image.zero_()              # the timed steps' survey image
    R.rbc_launch_count(reset=True)
    R.rbc_phase_timing(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record()
    for s in range(args.warmup, args.warmup + args.steps):
        flush.zero_()
        for shot in plan[s]:
            migrate(shot, seis[shot])
    reduce_image(image)        # Algorithm 3's stack over every rank's shots (no-op on one GPU)
    ev1.record()
    barrier()
    phases = R.rbc_phase_timing(ctx, False)
    launches = R.rbc_launch_count()
    clocks = smi.stop()
    el = ev0.elapsed_time(ev1) / 1e3
    if dist is not None:
        t = torch.tensor([el], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    shots_total = args.steps * B * world
    # Algorithm 3 solves three wave equations per step, Algorithm 2 two
    upd = (2 * w.npad * w.nt if storage else updates_per_shot(w)) * shots_total
    value = upd / el / 1e9

    # end to end: records from pinned host memory, image read back every step
    e2e = None
    if not args.no_e2e:
        host = {s: seis[s].cpu().pin_memory() for s in needed}
        stage = [torch.empty((nrec, w.nt + 1), dtype=torch.float32, device=dev) for _ in range(B)]
        img_host = torch.empty(g.interior, dtype=torch.float32).pin_memory()
        image.zero_()
        barrier()
        t0 = time.perf_counter()
        ev0.record()
        for s in range(args.warmup, args.warmup + args.steps):
            flush.zero_()
            for k, shot in enumerate(plan[s]):
                stage[k].copy_(host[shot], non_blocking=True)
                migrate(shot, stage[k])
            img_host.copy_(image, non_blocking=True)
        reduce_image(image)
        img_host.copy_(image, non_blocking=True)
        ev1.record()
        barrier()
        el_e2e = max(ev0.elapsed_time(ev1) / 1e3, 0.0)
        el_wall = time.perf_counter() - t0
        el_e2e = max(el_e2e, el_wall)
        if dist is not None:
            t = torch.tensor([el_e2e], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el_e2e = float(t.item())
        e2e = {"value": upd / el_e2e / 1e9, "unit": "Gpts/s",
               "h2d_bytes_per_step": B * nrec * (w.nt + 1) * 4,
               "d2h_bytes_per_step": int(image.numel()) * 4, "s_per_shot": el_e2e / (args.steps * B)}

    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    rev_launch_s = phases["rev_ms"] / 1e3 / max(phases["rev_launches"], 1)
    achieved = rev_bytes_per_launch(w) / rev_launch_s / 1e9
    fwd_launch_s = phases["fwd_ms"] / 1e3 / max(phases["fwd_launches"], 1)
    kname = "k_rev2d_tile" if w.ndim == 2 else "k_rev3d_tma"
    roofline = {"bound": "hbm", "kernel": f"{kname} (fused reverse pass)", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s",
                "traffic": (reverse_traffic(w.ndim, rev_bytes_per_launch(w))
                            if w.ndim == 3 or tuple(w.padded) == (871, 2421) else None),
                "traffic_source": ("ncu dram bytes of k_rev2d_tile on this grid, warm L2" if w.ndim == 2 else
                                   "ncu dram bytes of k_rev3d_tma on 380x380x280, scaled by the algorithmic bytes"),
                "bytes_per_launch": rev_bytes_per_launch(w), "launch_us": rev_launch_s * 1e6,
                "forward_kernel": {"kernel": "k_fwd2d" if w.ndim == 2 else "k_fwd3d_tma",
                                   "achieved": fwd_bytes_per_launch(w) / fwd_launch_s / 1e9,
                                   "launch_us": fwd_launch_s * 1e6,
                                   "bytes_per_launch": fwd_bytes_per_launch(w)},
                "note": ("one shot's working set (about 56 MB) is L2-resident during its time loop, "
                         "so achieved can exceed the HBM copy bandwidth") if w.ndim == 2 else
                        "working set of 4 GB: DRAM-bound"}

    if storage:
        nshots_ph = max(phases["shots"], 1)
        fb, rb = storage_phase_bytes(w, stride)
        fwd_s, rev_s = phases["fwd_ms"] / 1e3 / nshots_ph, phases["rev_ms"] / 1e3 / nshots_ph
        achieved = (fb + rb) / (fwd_s + rev_s) / 1e9
        roofline = {"bound": "hbm", "kernel": "k_fwd2d/k_fwd3d_tma steps + store/image kernels (whole phases)",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": roofline["peak_source"], "traffic": None,
                    "forward_phase": {"bytes": fb, "s": fwd_s, "GB/s": fb / fwd_s / 1e9},
                    "reverse_phase": {"bytes": rb, "s": rev_s, "GB/s": rb / rev_s / 1e9}}
    if rank != 0:
        R.rbc_destroy(ctx)
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1 and not storage:
        ns = ORACLE_SAMPLE_STEPS if w.ndim == 2 else 8
        v, dt = oracle_rtm_sample(w, inp, ns)
        cpu = {"value": v, "unit": "Gpts/s", "cores": cores_used(), "kind": "oracle",
               "sample": f"one full-grid shot ({'x'.join(map(str, w.padded[::-1]))} padded) of Algorithm 3 "
                         f"with {ns} of the {w.nt} time steps, {dt:.1f} s"}
    R.rbc_destroy(ctx)
    ctx = None
    shot3d = None
    if (args.workload == "survey2d" and not storage and world == 1 and not args.no_3d and not args.nt
            and not args.interior):
        del seis, num, den, flush
        torch.cuda.empty_cache()
        shot3d = shot3d_subrecord(R, W, torch, dev, peaks)
    out = {"metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "padded_grid": list(w.padded[::-1]), "nt": w.nt, "dt": w.dt,
                      "h": w.h, "receivers": nrec, "shots_per_step": B, "shots_timed": shots_total,
                      "s_per_shot": el / (args.steps * B),
                      "survey_s": el / (args.steps * B) * w.nshots,
                      "updates_per_shot": updates_per_shot(w),
                      "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                      "parallelism": f"shots sharded over {world} GPU(s)",
                      "method": (f"storage: Algorithm 2, source wavefield kept every {stride} steps "
                                 f"(Eq. 7, f_max = {2.5 * w.f_peak:g} Hz), store {store.numel() * 4 / 2**30:.2f} GiB "
                                 "in device memory") if storage else
                                "rbc: Algorithm 3, reconstruction through the random boundary"},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
           "clocks": clocks}
    if shot3d is not None:
        out["shot3d"] = shot3d
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
