"""The bench's unit arithmetic against the figures the workloads fix, and its
oracle (reference) leg, which runs on the host alone."""
import json
import os
import subprocess
import sys

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_updates_per_shot_match_the_workload_figures():
    # three leapfrog updates per padded node per step (forward, reconstruction,
    # receiver field), less the reconstruction's last level
    assert bench.updates_per_shot(W.SURVEY_2D) == 2421 * 871 * (3 * 12500 - 1)
    assert bench.updates_per_shot(W.SURVEY_2D) == pytest.approx(7.9e10, rel=0.01)
    assert bench.updates_per_shot(W.SHOT_3D) == pytest.approx(1.15e12, rel=0.01)


def test_algorithmic_bytes_per_launch():
    w = W.SURVEY_2D
    nint = w.nx * w.nz
    assert bench.fwd_bytes_per_launch(w) == 16 * w.npad
    assert bench.rev_bytes_per_launch(w) == 28 * w.npad + 16 * nint
    # an RTM step moves about 60 bytes per padded node for 3 updates
    per_node = (bench.fwd_bytes_per_launch(w) + bench.rev_bytes_per_launch(w)) / w.npad
    assert per_node == pytest.approx(60, rel=0.05)


def test_storage_phase_bytes():
    w = W.SHOT_3D
    k = 13
    f, r = bench.storage_phase_bytes(w, k)
    nint = w.nx * w.ny * w.nz
    kept = w.nt // k + 1
    assert f == 16 * w.npad * w.nt + 8 * nint * kept
    assert r == 16 * w.npad * w.nt + 24 * nint * kept


def test_shot_plan_covers_the_survey_once_per_pass():
    plan = bench.shot_plan(240, 30, 0, 8, 0, 1)
    flat = [s for step in plan for s in step]
    assert sorted(flat) == list(range(240))


def test_reference_leg_runs_on_the_host():
    """`bench.py --impl reference` times the FP64 oracle only: no GPU, one JSON line."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Gpts/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
