"""The benchmark's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

Under torchrun every rank advances its own independent lattice (no data-path collective); the
only cross-rank step is the max of the timed durations, from which rank 0 computes the whole-job
rate.  These tests run that logic with the gloo backend, and check that the reference arm does
its work on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [120.0, 80.0][rank]            # ms: rank 0 is the slower one
        e2e_s = [0.5, 0.9][rank]                 # s: rank 1 is the slower one
        t = bench.max_over_ranks(elapsed, dist, "cpu")
        te = bench.max_over_ranks(e2e_s, dist, "cpu")
        out[rank] = (t, te, bench.job_rate(world, 1000, 10, t * 1e-3), bench.replica_seed(rank))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo_world2():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 120.0
    assert out[0][1] == out[1][1] == 0.9
    assert out[0][2] == pytest.approx(2 * 1000 * 10 / 0.12)
    assert out[0][3] != out[1][3]                # independent replicas


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(1, 100, 4, 2.0) == 200.0


def test_reference_arm_other_ranks_do_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_recorded_counters_follow_the_kernel_source(monkeypatch):
    """The ncu per-site figures apply only to the kernel source they were taken on."""
    import json
    with open(os.path.join(ROOT, "profiles", "step2d_f32_traffic.json")) as f:
        d = json.load(f)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda precision=32: d["kernel_source_hash"])
    a = bench.alu_roofline(4096 * 4096, 0.9, 152)
    assert a["bound"] == "alu" and 0 < a["frac"] < 1.2
    assert a["frac"] == pytest.approx(d["fma_pipe_cycles_per_site"] * 4096 * 4096 / 0.9e-3 / a["peak"])
    assert bench.recorded_traffic(4096) == pytest.approx(d["dram_bytes_per_site"] * 4096 * 4096)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda precision=32: "0" * 16)
    assert bench.recorded_traffic(4096) is None
    assert bench.alu_roofline(4096 * 4096, 0.9, 152)["frac"] is None
