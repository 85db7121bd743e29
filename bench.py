#!/usr/bin/env python
"""Throughput of the spin-2 QLGA step on GB300: site-updates/s and fraction of the HBM roofline.

Workload (one "step" = one QLGA time step: potential unitary + kinetic operator on both axes,
with the FP64 observables every --obs-every steps): the 2D vortex-scattering lattice, 4096 x 4096
sites, 10 FP32 amplitudes per site, Pade vortex dipoles in m = +2 / -2, couplings (1, 0.1, 1),
eps = 0.1.  The state (1.34 GB) is larger than L2, so no flush is needed between steps.

The lattice is first evolved --settle steps untimed (default 1000): the vortex background is
dynamically unstable, and within ~1000 steps the whole lattice fills with structure, the two
qubits of a pair drift apart and the potential needs its full Taylor degree on both of its
vectors.  The first few hundred steps run up to 30% faster, so timing them would overstate the
rate of the 5000-step run.

  python bench.py [--gpus N --steps K --warmup W]            # the library (default)
  python bench.py --impl reference                           # the FP64 CPU oracle, same metric

Multi-GPU (torchrun): every rank advances its own independent lattice (a replica with its own
seed); there is no data-path collective, so scaling is weak and value = all ranks' site-updates
over the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QLGA site-updates/s and % of HBM roofline (FP32 vs FP64, plain vs batched/adjoint)"
UNIT = "site-updates/s"
BYTES_PER_SITE_F32 = 160      # one read + one write of 10 complex FP32 amplitudes
FIELDS_BYTES_PER_SITE_F32 = 80 + 44   # qlga_fields: one read of the true state, 11 FP32 values written


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=4096, help="lattice side")
    p.add_argument("--precision", type=int, default=32, choices=[32, 64],
                   help="state precision of the timed lattice (64: the FP64 path of the same workload)")
    p.add_argument("--obs-every", type=int, default=50)
    p.add_argument("--settle", type=int, default=1000, help="untimed steps before the warm-up")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-paths", action="store_true",
                   help="skip the FP64 / batched / adjoint / interleaved comparison runs")
    p.add_argument("--no-accuracy", action="store_true",
                   help="skip the paths' accuracy runs against the stored oracle results")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(rank):
    """Each rank advances its own independent lattice: config 2's seed offset by the rank."""
    return 1909 + rank


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, sites, steps, seconds):
    """Whole-job rate: the site-updates of all ranks over the slowest rank's time."""
    return world * sites * steps / seconds


# ----------------------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f",
                                          self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != self.gpu:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def strip_comments(src):
    """C++ source without its comments and trailing blanks: what the compiler sees of it (the
    kernel sources hold no string literal with a comment marker)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


STEP_SOURCES = {32: ("qlga_step2d.cuh", "qlga_device.cuh"),
                64: ("qlga_step2d_f64.cuh", "qlga_interleave.cuh", "qlga_step2d.cuh", "qlga_device.cuh")}
STEP_COUNTERS = {32: "step2d_f32_traffic.json", 64: "step2d_f64_counters.json"}


def kernel_source_hash(precision=32):
    """Hash of the fused step kernel's sources, comments excluded: the committed ncu figures stay
    valid across comment edits and lapse with any change to the code."""
    h = hashlib.sha256()
    for name in STEP_SOURCES[precision]:
        with open(os.path.join(ROOT, "paper_1907_12834_gb300", "csrc", name)) as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_step_counters(precision=32):
    """The committed ncu figures of the fused step kernel (per site), or None when the summary is
    missing or the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", STEP_COUNTERS[precision])
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    return d if d.get("kernel_source_hash") == kernel_source_hash(precision) else None


def counters_note():
    """One line from the committed ncu figures of the fused step, if they match the source."""
    d = recorded_step_counters()
    if d is None:
        return "no ncu figure for the current kernel source"
    return "FMA pipe %.0f%% busy, %.1f DRAM bytes per site against %d algorithmic" % (
        100 * float(d["fma_pipe_busy_frac"]), float(d["dram_bytes_per_site"]),
        int(d["algorithmic_bytes_per_site"]))


def alu_roofline(sites, kernel_ms, sms):
    """FP32 FMA-pipe view of the fused step: issue cycles per site from the ncu capture, over the
    live launch duration, against one FMA-pipe issue per SM sub-partition per cycle at the maximum
    SM clock (4 sub-partitions per SM)."""
    d = recorded_step_counters()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, KeyError, ValueError):
        mhz, src = 2070.0, "nominal 2070 MHz"
    peak = 4.0 * sms * mhz * 1e6
    if d is None or "fma_pipe_cycles_per_site" not in d:
        return {"bound": "alu", "achieved": None, "peak": peak, "unit": "FMA-pipe issue cycles/s",
                "frac": None, "note": "no ncu figure for the current kernel source"}
    per_site = float(d["fma_pipe_cycles_per_site"])
    achieved = per_site * sites / (kernel_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "FMA-pipe issue cycles/s",
            "frac": achieved / peak, "cycles_per_site": per_site,
            "peak_source": "4 sub-partitions x %d SMs x %s" % (sms, src),
            "note": "FP32 FMA-pipe issue cycles per site from an ncu --set full capture of the fused "
                    "step on the settled 2048^2 state; the pipe, not HBM, bounds the fused step"}


def recorded_traffic(n, precision=32):
    """DRAM bytes per launch of the fused step kernel from the committed ncu summary, scaled to an
    n x n lattice; None when the summary is missing or the kernel source changed since."""
    d = recorded_step_counters(precision)
    return None if d is None else float(d["dram_bytes_per_site"]) * n * n


def alu64_roofline(sites, kernel_ms, sms):
    """FP64-pipe view of the fused FP64 step, by the method of alu_roofline: FP64-pipe cycles per
    site from the ncu capture (pct of peak sustained active x smsp__cycles_active.sum / sites)
    over the live launch duration, against one FP64-pipe cycle per SM sub-partition per cycle at
    the maximum SM clock; beside it the FP64 arithmetic rate (DFMA = 2 flops) against the nominal
    1.25 TFLOP/s of GB300."""
    d = recorded_step_counters(64)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, KeyError, ValueError):
        mhz, src = 2070.0, "nominal 2070 MHz"
    peak = 4.0 * sms * mhz * 1e6
    if d is None or "fp64_pipe_cycles_per_site" not in d:
        return {"bound": "alu", "achieved": None, "peak": peak, "unit": "FP64-pipe cycles/s",
                "frac": None, "note": "no ncu figure for the current kernel source"}
    per_site = float(d["fp64_pipe_cycles_per_site"])
    achieved = per_site * sites / (kernel_ms * 1e-3)
    flops = float(d["fp64_flops_per_site"]) * sites / (kernel_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "FP64-pipe cycles/s",
            "frac": achieved / peak, "cycles_per_site": per_site,
            "peak_source": "4 sub-partitions x %d SMs x %s" % (sms, src),
            "fp64_tflops": flops / 1e12, "fp64_nominal_tflops": 1.25,
            "fp64_frac_of_nominal": flops / 1.25e12,
            "note": "FP64-pipe cycles and FP64 operations per site from an ncu capture of the fused "
                    "FP64 step on the settled 2048^2 state"}


def cpu_baseline(state_f64, g, budget_s, n_sub=256):
    """The oracle as it stands, on a bounded sample: an n_sub^2 window of the workload."""
    import numpy as np
    import oracle

    cores = os.cpu_count() or 1
    ny, nx = state_f64.shape[1], state_f64.shape[2]
    y0, x0 = ny // 2 - n_sub // 2, nx // 2 - n_sub // 2
    win = np.ascontiguousarray(state_f64[:, y0:y0 + n_sub, x0:x0 + n_sub], dtype=np.float64)
    cfg = oracle.make_cfg(2, n_sub, n_sub, *g)
    t0 = time.perf_counter()
    oracle.step(win, cfg, 1, nthreads=cores)
    t1 = time.perf_counter()
    steps = max(1, min(200, int(budget_s / max(t1 - t0, 1e-6))))
    t0 = time.perf_counter()
    oracle.step(win, cfg, steps, nthreads=cores)
    dt = time.perf_counter() - t0
    # the same oracle on one core, a 64 x 64 window of the same state, about 3 s
    n1 = 64
    win1 = np.ascontiguousarray(win[:, :n1, :n1])
    cfg1 = oracle.make_cfg(2, n1, n1, *g)
    t0 = time.perf_counter()
    oracle.step(win1, cfg1, 1, nthreads=1)
    s1 = max(1, min(100, int(3.0 / max(time.perf_counter() - t0, 1e-6))))
    t0 = time.perf_counter()
    oracle.step(win1, cfg1, s1, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": n_sub * n_sub * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d x %d window at the lattice centre of the same workload, %d FP64 steps, "
                      "%.1f s" % (n_sub, n_sub, steps, dt),
            "single_core": {"value": n1 * n1 * s1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": "%d x %d window of the same state, %d FP64 steps, %.1f s" % (n1, n1, s1, dt1)}}


# ----------------------------------------------------------------------------- library arm

def run_gb300(args):
    import numpy as np
    import torch

    from paper_1907_12834_gb300 import inputs, qlga

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    f64 = args.precision == 64
    w = inputs.config2(seed=replica_seed(rank), n=n, dtype=np.float64 if f64 else np.float32)
    lat = qlga.Lattice(2, n, n, precision=args.precision, g=w.g, epsilon=w.eps)
    stream = lat.stream
    sites = n * n

    lat.load_state(w.state)
    if args.settle:
        lat.step(args.settle)
    settled = w.state if not args.settle else lat.get_state()
    lat.load_state(settled)
    lat.step(args.warmup)
    obs0 = lat.observables()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = lat.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    obs_steps = set()
    ev[0].record(stream)
    for i in range(args.steps):
        lat.step(1)
        if args.obs_every and (i + 1) % args.obs_every == 0:
            lat.observables()               # FP64 reductions, host read
            obs_steps.add(i)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    launches = lat.launch_count() - launches0
    obs1 = lat.observables()
    drift = {"norm_qubit_rel": abs(obs1["norm_qubit"] - obs0["norm_qubit"]) / obs0["norm_qubit"],
             "energy_rel": abs(obs1["energy"] - obs0["energy"]) / abs(obs0["energy"]),
             "steps": args.steps,
             "note": "%s state, FP64 sums, over the timed steps; the qubit norm is conserved exactly by "
                     "every step, so its drift is rounding; the energy of the discretised field is "
                     "not an exact invariant of the QLGA step" % ("FP64" if f64 else "FP32")}
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None

    elapsed_ms = ev[0].elapsed_time(ev[args.steps])
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    plain = [t for i, t in enumerate(step_ms) if i not in obs_steps] or step_ms
    kernel_ms = statistics.mean(plain)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(lat, settled, args, torch, qlga, sites)
        e2e["value"] = job_rate(world, sites, args.steps, max_over_ranks(e2e.pop("seconds"), dist, "cuda"))
    lat.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    bytes_per_site = 2 * BYTES_PER_SITE_F32 if f64 else BYTES_PER_SITE_F32
    achieved = bytes_per_site * sites / (kernel_ms * 1e-3) / 1e9
    traffic = recorded_traffic(n, 64 if f64 else 32)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    line = {
        "metric": METRIC, "value": job_rate(world, sites, args.steps, elapsed_ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if f64 else "f32", "data": "synthetic (seeded Pade vortex dipoles)",
        "config": {"workload": w.name, "lattice": [n, n], "precision": "fp64" if f64 else "fp32",
                   "couplings": list(w.g), "epsilon": w.eps, "obs_every": args.obs_every,
                   "timed_after_step": args.settle + args.warmup,
                   "l2": "inputs larger than L2 (%.2f GB state)" % (sites * (160 if f64 else 80) / 1e9),
                   "parallelism": "replicas%d" % world},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "kernel_ms": kernel_ms, "algorithmic_bytes_per_site": bytes_per_site,
                     "note": ("the FP64 step is bound by the FP64 pipe (see alu)" if f64 else
                              "the fused step is limited by FP32 FMA-pipe cycles of the potential "
                              "(ncu --set full on the settled 2048^2 state: %s), "
                              "not by HBM traffic" % counters_note())},
        "alu": alu64_roofline(sites, kernel_ms, sms) if f64 else alu_roofline(sites, kernel_ms, sms),
        "e2e": e2e,
        "drift": drift,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_paths and not f64:
        # the FP64 and interleaved comparisons start from the settled state the headline is timed on
        line["paths"] = run_paths(args, torch, qlga, inputs, settled.astype(np.float32), line["value"] / world)
        lh = line["paths"].get("long_horizon", {}).get("config2_512")
        if lh:
            # the timed kernel's own accuracy: the same fused FP32 step on the config 2 recipe at
            # 512^2 against the FP64 oracle, at each checkpoint of config 2's 5000 steps
            line["accuracy"] = {"workload": "config2_512", "steps": lh["steps"],
                                "gpu_fp32_vs_oracle": lh["gpu_fp32_vs_oracle"],
                                "gpu_fp64_vs_oracle": lh["gpu_fp64_vs_oracle"],
                                "oracle_perturbed_1e-13": lh["oracle_perturbed_1e-13"],
                                "note": "relative L2 at the stored sample of sites; the last column shows "
                                        "how the dynamics amplifies a 1e-13 change of the initial state"}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w.state, w.g, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _timed_steps(torch, lat, steps):
    """Device time per step of `steps` plain steps on the lattice's stream (after a warm-up)."""
    lat.step(2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / steps


def run_paths(args, torch, qlga, inputs, state_f32, rate_fp32):
    """The comparisons the metric names, each timed on the device after a warm-up: the plain
    step in FP64 on the same lattice, the batched 1D path against one FP64 run at a time, the
    adjoint (checkpointed forward + pull-back) against the plain FP64 step on its lattice, and the
    interleaved step.  Accuracy of each path against the FP64 oracle is established by the
    parity tests (FP64 1e-11, FP32 1e-5 per configuration)."""
    import numpy as np
    out = {}
    n = args.n
    # plain FP64 on the bench lattice (same initial data)
    lat = qlga.Lattice(2, n, n, precision=64, g=inputs.CONFIG2_G)
    lat.load_state(state_f32.astype(np.float64))
    sec = _timed_steps(torch, lat, 3)
    lat.close()
    out["plain_fp64_2d"] = {"lattice": [n, n], "site_updates_per_s": n * n / sec, "ms_per_step": sec * 1e3,
                            "alu": alu64_roofline(n * n, sec * 1e3,
                                                  torch.cuda.get_device_properties(0).multi_processor_count)}
    out["fp32_over_fp64_2d"] = rate_fp32 / out["plain_fp64_2d"]["site_updates_per_s"]
    # plain 1D single lattices: config 1 (two-soliton scattering, 16384 sites) in FP32 and FP64,
    # config 0 (bright soliton, 1024 sites) in FP64 -- latency-bound sizes, stepped through graphs
    def rate_1d(w, precision, steps):
        lat = qlga.Lattice(1, w.nx, 1, precision=precision, g=w.g, epsilon=w.eps)
        lat.load_state(w.state.astype(np.float32 if precision == 32 else np.float64))
        lat.step(100)                                   # shape tuning, graph capture
        sec = _timed_steps(torch, lat, steps)
        shape = lat.shape_1d()
        lat.close()
        return {"lattice": w.nx, "site_updates_per_s": w.nx / sec, "us_per_step": sec * 1e6,
                "shape": list(shape)}
    c1 = inputs.config1()
    out["config1_fp32_1d"] = rate_1d(c1, 32, 2000)
    out["config1_fp64_1d"] = rate_1d(c1, 64, 500)
    out["config0_fp64_1d"] = rate_1d(inputs.config0(), 64, 2000)
    # interleaved FP32 on the bench lattice
    lat = qlga.Lattice(2, n, n, precision=32, g=inputs.CONFIG2_G, interleave=1)
    lat.load_state(state_f32)
    sec = _timed_steps(torch, lat, 10)
    lat.close()
    out["interleaved_fp32_2d"] = {"lattice": [n, n], "site_updates_per_s": n * n / sec, "ms_per_step": sec * 1e3}
    # per-site diagnostic fields of the bench lattice (F_par, F_perp, |A00|, colour map, vorticity
    # of each level): one read of the true state (80 B per site in FP32) and 11 values written per
    # site (44 B), on the device
    lat = qlga.Lattice(2, n, n, precision=32, g=inputs.CONFIG2_G)
    lat.load_state(state_f32)
    fbuf = torch.empty(11 * n * n, dtype=torch.float32, device="cuda")
    qlga.qlga_fields(lat.handle, fbuf.data_ptr(), qlga.QLGA_DEVICE)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    for _ in range(10):
        qlga.qlga_fields(lat.handle, fbuf.data_ptr(), qlga.QLGA_DEVICE)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    lat.close()
    del fbuf
    peak, peak_kind = measured_peaks()
    gbs = FIELDS_BYTES_PER_SITE_F32 * n * n / (ms * 1e-3) / 1e9
    out["fields_fp32_2d"] = {"lattice": [n, n], "ms_per_call": ms, "sites_per_s": n * n / (ms * 1e-3),
                             "algorithmic_bytes_per_site": FIELDS_BYTES_PER_SITE_F32, "achieved_gbs": gbs,
                             "hbm_frac": gbs / peak, "peak_source": peak_kind,
                             "accuracy": "against the oracle's fields in the GPU parity tests"}
    # batched 1D (256 runs, FP32, graph replay) against one FP64 run of the mean length
    bw = inputs.config3()
    b = qlga.Batch1D(bw.lengths, bw.couplings, precision=32)
    b.load_state(bw.state)
    b.step(20)                                   # tuner + graph capture
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(200)
    e1.record(b.stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3 / 200
    total = int(bw.lengths.sum())
    info = b.info()
    b.close()
    L = int(round(float(bw.lengths.mean())))
    rng = np.random.default_rng(1910)
    one = inputs.boson_to_state(inputs.scattering_run(rng, L, bw.eps), bw.eps)
    lat = qlga.Lattice(1, L, 1, precision=64, g=tuple(bw.couplings[0]))
    lat.load_state(one)
    sec1 = _timed_steps(torch, lat, 200)
    lat.close()
    out["batched_fp32_1d"] = {"runs": int(len(bw.lengths)), "sites": total, "site_updates_per_s": total / sec,
                              "ms_per_step": sec * 1e3, "tile_width": info["tile_width"],
                              "sites_per_thread": info["sites_per_thread"],
                              "steps_per_launch": info["steps_per_launch"]}
    out["single_run_fp64_1d"] = {"lattice": L, "site_updates_per_s": L / sec1, "ms_per_step": sec1 * 1e3}
    out["batched_fp32_over_single_run_fp64"] = (total / sec) / (L / sec1)
    # batched 2D (128 runs of 64..512 x 64..512 sites, FP32) against one FP64 run of the batch
    b2 = inputs.batch2d()
    heights = b2.meta["heights"]
    b = qlga.Batch(b2.lengths, b2.couplings, precision=32, heights=heights)
    b.load_state(b2.state)
    b.step(20)
    torch.cuda.synchronize()
    e0.record(b.stream)
    b.step(100)
    e1.record(b.stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3 / 100
    total2 = int((b2.lengths * heights).sum())
    b.close()
    r0 = int(np.argsort(b2.lengths * heights)[len(heights) // 2])   # the run of median size
    o0 = int(20 * (b2.lengths[:r0] * heights[:r0]).sum())
    nx0, ny0 = int(b2.lengths[r0]), int(heights[r0])
    lat = qlga.Lattice(2, nx0, ny0, precision=64, g=tuple(b2.couplings[r0]))
    lat.load_state(b2.state[o0:o0 + 20 * nx0 * ny0].reshape(5, ny0, nx0, 2, 2).astype(np.float64))
    sec1 = _timed_steps(torch, lat, 20)
    lat.close()
    out["batched_fp32_2d"] = {"runs": int(len(heights)), "sites": total2, "site_updates_per_s": total2 / sec,
                              "ms_per_step": sec * 1e3}
    out["single_run_fp64_2d"] = {"lattice": [nx0, ny0], "site_updates_per_s": nx0 * ny0 / sec1,
                                 "ms_per_step": sec1 * 1e3}
    out["batched_fp32_2d_over_single_run_fp64"] = (total2 / sec) / (nx0 * ny0 / sec1)
    # adjoint on the 512^2 lattice: 200 steps forward with checkpoints every 100, then the pull-back
    for prec in (32, 64):
        w4 = inputs.config4(dtype=np.float32 if prec == 32 else np.float64)
        dt = torch.float32 if prec == 32 else torch.float64
        x0 = torch.tensor(w4.state, dtype=dt, device="cuda")
        lat = qlga.Lattice(2, 512, 512, precision=prec, g=w4.g)
        steps, C = 200, 100
        ws = lat.adjoint_workspace(steps, C)
        lat.adjoint_forward(x0, steps, C, ws)        # warm-up
        lat.adjoint_backward(x0, steps, C, ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.adjoint_forward(x0, steps, C, ws)
        xn = lat.device_state()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        cot, _ = lat.adjoint_backward(xn, steps, C, ws)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        err = float(torch.linalg.vector_norm((cot - x0).double()) / torch.linalg.vector_norm(x0.double()))
        plain = None
        if prec == 64:
            lat.load_state(x0)
            plain = 512 * 512 / _timed_steps(torch, lat, 10)
        lat.close()
        del ws
        sites = 512 * 512
        out["adjoint_fp%d_2d_512" % prec] = {
            "steps": steps, "checkpoint_every": C,
            "gradient_site_steps_per_s": sites * steps / (t2 - t0),
            "forward_ms_per_step": (t1 - t0) * 1e3 / steps, "backward_ms_per_step": (t2 - t1) * 1e3 / steps,
            "norm_identity_error": err}
        if plain:
            out["plain_fp64_2d_512"] = {"site_updates_per_s": plain}
    out["adjoint_fp32_over_plain_fp64_2d_512"] = (out["adjoint_fp32_2d_512"]["gradient_site_steps_per_s"] /
                                                 out["plain_fp64_2d_512"]["site_updates_per_s"])
    out["note"] = ("rates on the device with CUDA events (adjoint: wall time of the two calls, host "
                   "synchronised); gradient_site_steps_per_s counts sites x steps of a full gradient "
                   "(forward with checkpoints + recompute + pull-back); norm_identity_error = "
                   "|dL/dx0 - x0| / |x0| for L = |x_n|^2 / 2; 'accuracy' of a path: its kernels run "
                   "on a short case of the path's recipe against the FP64 oracle's stored results")
    if args.no_accuracy:
        return out
    acc = path_accuracy(torch, qlga, inputs) or {}
    lh = long_horizon_record(torch, qlga, inputs)
    for key, src in (("config0_fp64_1d", "config0_fp64_1d"), ("interleaved_fp32_2d", "interleaved_fp32_2d"),
                     ("batched_fp32_1d", "batched_fp32_1d"), ("batched_fp32_2d", "batched_fp32_2d"),
                     ("adjoint_fp32_2d_512", "adjoint_fp32_2d"), ("adjoint_fp64_2d_512", "adjoint_fp64_2d")):
        if src in acc and key in out:
            out[key]["accuracy"] = acc[src]
    for key, prec, name in (("config1_fp32_1d", 32, "config1_g_integrable_set"),
                            ("config1_fp64_1d", 64, "config1_g_integrable_set"),
                            ("plain_fp64_2d", 64, "config2_512")):
        if name in lh and key in out:
            r = lh[name]
            out[key]["accuracy"] = {"workload": name, "steps": r["steps"][-1],
                                    "rel_l2_vs_oracle": r["gpu_fp%d_vs_oracle" % prec][-1],
                                    "oracle_perturbed_1e-13": r["oracle_perturbed_1e-13"][-1],
                                    "norm_drift": r["gpu_fp%d_norm_drift" % prec]}
    out["long_horizon"] = lh
    return out


GOLDEN = os.path.join(ROOT, "tests", "golden")


def _rel(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _sample(state, sites):
    """The state (library layout) at flat site indices: (5, len(sites), 2, 2)."""
    return state.reshape(5, -1, 2, 2)[:, sites]


def long_horizon_record(torch, qlga, inputs, names=None):
    """GPU FP64 and FP32 runs of the long-horizon workloads against the FP64 oracle's stored
    trajectory (tests/golden/long_horizon_*.npz, written by a script that calls only the oracle),
    every checkpoint: relative L2 at the stored sample of sites; beside them the growth of a
    1e-13 relative perturbation of the initial state, in the oracle (stored) and in the GPU FP64
    run (full lattice), which shows how far the dynamics itself amplifies rounding."""
    import numpy as np
    out = {}
    for name in names or inputs.LONG_HORIZON:
        path = os.path.join(GOLDEN, "long_horizon_%s.npz" % name)
        if not os.path.exists(path):
            continue
        G = np.load(path)
        ndim, nx, ny, g, steps, every, x0 = inputs.long_horizon_workload(name)
        rec = {"lattice": [nx, ny] if ndim == 2 else nx, "couplings": list(g),
               "steps": [int(k) for k in G["steps"]], "oracle_perturbed_1e-13": [float(v) for v in G["oracle_growth"]]}
        for prec in (64, 32):
            dt = np.float64 if prec == 64 else np.float32
            lat = qlga.Lattice(ndim, nx, ny, precision=prec, g=g)
            lat.load_state(x0.astype(dt))
            latp = None
            if prec == 64:
                latp = qlga.Lattice(ndim, nx, ny, precision=prec, g=g)
                latp.load_state(inputs.perturbed(x0))
            errs, growth, norm = [], [], []
            for k, step in enumerate(G["steps"]):
                if step > 0:
                    lat.step(every)
                    if latp is not None:
                        latp.step(every)
                st = lat.get_state()
                errs.append(_rel(_sample(st, G["sites"][k]), G["samples"][k]))
                norm.append(float((st.astype(np.float64) ** 2).sum()))
                if latp is not None:
                    growth.append(_rel(latp.get_state(), st))
            lat.close()
            if latp is not None:
                latp.close()
                rec["gpu_fp64_perturbed_1e-13"] = growth
            rec["gpu_fp%d_vs_oracle" % prec] = errs
            rec["gpu_fp%d_norm_drift" % prec] = abs(norm[-1] - norm[0]) / norm[0]
        out[name] = rec
    return out


def path_accuracy(torch, qlga, inputs):
    """Each timed path run on a short case of its own recipe and compared with the FP64 oracle's
    stored results (tests/golden/path_accuracy.npz): relative L2 at the stored sites (whole state
    for config 0), with the qubit-norm drift of the run."""
    import numpy as np
    path = os.path.join(GOLDEN, "path_accuracy.npz")
    if not os.path.exists(path):
        return None
    G = np.load(path)
    W = inputs.path_accuracy_workloads()
    out = {}

    def lattice_run(w, prec, steps, interleave=0):
        lat = qlga.Lattice(w.ndim, w.nx, w.ny, precision=prec, g=w.g, interleave=interleave)
        lat.load_state(w.state.astype(np.float32 if prec == 32 else np.float64))
        n0 = lat.observables()["norm_qubit"]
        lat.step(steps)
        o = lat.observables()
        st = lat.get_state()
        lat.close()
        return st, abs(o["norm_qubit"] - n0) / n0

    c = W["config0"]
    st, dn = lattice_run(c["w"], 64, c["steps"])
    out["config0_fp64_1d"] = {"steps": c["steps"], "rel_l2_vs_oracle": _rel(st, G["config0_state"]),
                              "norm_drift": dn}
    c = W["interleaved"]
    st, dn = lattice_run(c["w"], 32, c["steps"], interleave=1)
    out["interleaved_fp32_2d"] = {"lattice": [c["w"].nx, c["w"].ny], "steps": c["steps"],
                                  "rel_l2_vs_oracle": _rel(_sample(st, G["interleaved_sites"]),
                                                           G["interleaved_samples"]), "norm_drift": dn}
    for key, heights_of in (("batch1d", None), ("batch2d", "heights")):
        c = W[key]
        b = c["w"]
        hs = b.meta["heights"] if heights_of else np.ones(len(b.lengths), dtype=np.int64)
        kw = {"heights": hs} if heights_of else {}
        bt = qlga.Batch(b.lengths, b.couplings, precision=32, **kw)
        bt.load_state(b.state.astype(np.float32))
        bt.step(c["steps"])
        got = bt.get_state().astype(np.float64)
        bt.close()
        sizes = b.lengths * hs
        offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        sites = G[key + "_sites"]
        run = np.searchsorted(offs, sites, side="right") - 1
        gs = np.empty((5, len(sites), 2, 2))
        for r in np.unique(run):
            sel = run == r
            part = got[20 * offs[r]:20 * (offs[r] + sizes[r])].reshape(5, -1, 2, 2)
            gs[:, sel] = part[:, sites[sel] - offs[r]]
        n0 = float((b.state.astype(np.float64) ** 2).sum())
        out["batched_fp32_%s" % key[-2:]] = {"runs": int(len(b.lengths)), "steps": c["steps"],
                                            "rel_l2_vs_oracle": _rel(gs, G[key + "_samples"]),
                                            "norm_drift": abs(float((got ** 2).sum()) - n0) / n0}
    c = W["adjoint"]
    w4 = c["w"]
    for prec in (32, 64):
        dt = torch.float32 if prec == 32 else torch.float64
        x0 = torch.tensor(w4.state, dtype=dt, device="cuda")
        cot_in = torch.tensor(inputs.adjoint_cotangent(w4.state.shape, c["cotangent_seed"]), dtype=dt, device="cuda")
        with qlga.Lattice(2, w4.nx, w4.ny, precision=prec, g=w4.g) as lat:
            cot, dg = lat.gradient(x0, c["steps"], cot_in, checkpoint_every=30)
        cn = cot.double().cpu().numpy()
        out["adjoint_fp%d_2d" % prec] = {
            "lattice": [w4.nx, w4.ny], "steps": c["steps"],
            "rel_l2_vs_oracle": _rel(_sample(cn, G["adjoint_sites"]), G["adjoint_cot_samples"]),
            "coupling_gradient_rel_vs_oracle": float(np.abs(np.asarray(dg) - G["adjoint_dg"]).max() /
                                                     np.abs(G["adjoint_dg"]).max())}
    return out


E2E_REPEATS = 3


def run_e2e(lat, state, args, torch, qlga, sites):
    """Same steps through the C ABI with host buffers: pinned upload of the (settled) state,
    steps, observables, pinned read-back of the final state, all inside the timed region.  The
    pinned copies share the host's memory with other work on the machine, so the run is made
    E2E_REPEATS times and the median time is reported (all of them are listed)."""
    host_in = torch.from_numpy(state).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    times, phases = [], []
    for _ in range(E2E_REPEATS):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qlga.qlga_load_state(lat.handle, host_in.data_ptr(), qlga.QLGA_HOST)
        t1 = time.perf_counter()
        for i in range(args.steps):
            qlga.qlga_step(lat.handle, 1)
            if args.obs_every and (i + 1) % args.obs_every == 0:
                qlga.qlga_observables(lat.handle)
        t2 = time.perf_counter()
        qlga.qlga_get_state(lat.handle, host_out.data_ptr(), qlga.QLGA_HOST)
        t3 = time.perf_counter()
        times.append(t3 - t0)
        phases.append({"upload_ms": (t1 - t0) * 1e3, "steps_ms": (t2 - t1) * 1e3, "read_back_ms": (t3 - t2) * 1e3})
    dt = sorted(times)[len(times) // 2]
    nbytes = host_in.numel() * host_in.element_size()
    return {"value": sites * args.steps / dt, "unit": UNIT, "seconds": dt,
            "repeats": [sites * args.steps / t for t in times], "phases": phases,
            "h2d_bytes_per_step": nbytes / args.steps,
            "d2h_bytes_per_step": (nbytes + 8 * 16 * (args.steps // max(args.obs_every, 1))) / args.steps,
            "note": "the simulation's input is its state: uploaded once from pinned host memory, "
                    "%d steps with the observables read back every %d steps, the final state read "
                    "back to pinned memory; bytes per step = those transfers / steps; median of %d "
                    "runs (repeats)" % (args.steps, args.obs_every, E2E_REPEATS)}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 CPU oracle, as it stands, on this host's cores: each step advances a bounded
    sample (a 256^2 window) of the same workload by one QLGA step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1907_12834_gb300 import inputs

    n_sub = 256
    w = inputs.config2(n=args.n)
    ny = nx = args.n
    y0, x0 = ny // 2 - n_sub // 2, nx // 2 - n_sub // 2
    win = np.ascontiguousarray(w.state[:, y0:y0 + n_sub, x0:x0 + n_sub], dtype=np.float64)
    del w
    cfg = oracle.make_cfg(2, n_sub, n_sub, *inputs.CONFIG2_G)
    cores = os.cpu_count() or 1
    oracle.step(win, cfg, args.warmup, nthreads=cores)
    t0 = time.perf_counter()
    oracle.step(win, cfg, args.steps, nthreads=cores)
    dt = time.perf_counter() - t0
    value = n_sub * n_sub * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Pade vortex dipoles)",
        "config": {"workload": "2d-vortex-scattering-%dx%d" % (args.n, args.n),
                   "lattice": [args.n, args.n], "precision": "fp64 (oracle)",
                   "couplings": list(inputs.CONFIG2_G), "epsilon": 0.1,
                   "sample": "%d x %d window per step" % (n_sub, n_sub)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d x %d window of the workload, %d steps" % (n_sub, n_sub, args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
