"""Writes tests/golden/path_accuracy.npz: the FP64 oracle's results for one short run of each
path the benchmark times, the expected values against which each path's accuracy is stated.

Calls only the oracle (oracle/) and the seeded input generators (paper_1907_12834_gb300.inputs).
Each workload is a small case of the path's own recipe; states are stored at a sample of sites
(the densest 3/4 and a seeded uniform draw of the rest, as in make_long_horizon.py), or whole
when small:
  config0     config 0 (Table I row 1 bright soliton, L = 1024), 2000 plain steps, whole state
  interleaved the config 2 recipe on 128^2, 100 interleaved steps (U^(1/8) before each block)
  batch1d     6 runs of the config 3 recipe with L log-uniform in [512, 2048], 500 steps each
              under the run's couplings
  batch2d     the first 4 runs of the 2D batch recipe, 100 steps each
  adjoint     the config 4 recipe on 64^2 (cores 20 apart), 100 steps: dL/dx0 and dL/dg of
              L = <w, x_100> for a seeded w (the oracle's pull-back, vjp_run)

  python tests/golden/make_path_accuracy.py [--threads N]
"""
import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1907_12834_gb300 import inputs  # noqa: E402


def sample_sites(x, nsites, count, seed):
    dens = (x.reshape(5, nsites, 4) ** 2).sum(axis=(0, 2))
    count = min(count, nsites)
    ntop = (3 * count) // 4
    top = np.argsort(-dens, kind="stable")[:ntop]
    rest = np.setdiff1d(np.arange(nsites), top)
    extra = np.random.default_rng(seed).choice(rest, size=count - ntop, replace=False)
    return np.sort(np.concatenate([top, extra]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    th = ap.parse_args().threads
    W = inputs.path_accuracy_workloads()
    out = {}

    c = W["config0"]
    w = c["w"]
    x = np.ascontiguousarray(w.state, dtype=np.float64)
    oracle.step(x, oracle.make_cfg(1, w.nx, 1, *w.g), c["steps"], th)
    out["config0_steps"] = c["steps"]
    out["config0_state"] = x

    c = W["interleaved"]
    w = c["w"]
    x = np.ascontiguousarray(w.state)
    oracle.step(x, oracle.make_cfg(2, w.nx, w.ny, *w.g, interleave=c["interleave"]), c["steps"], th)
    idx = sample_sites(x, w.nx * w.ny, 1024, 1)
    out["interleaved_steps"] = c["steps"]
    out["interleaved_sites"] = idx
    out["interleaved_samples"] = x.reshape(5, -1, 2, 2)[:, idx]

    c = W["batch1d"]
    b = c["w"]
    offs = np.concatenate([[0], np.cumsum(b.lengths)[:-1]])
    sites, samples = [], []
    for r, L in enumerate(b.lengths):
        L = int(L)
        x = np.ascontiguousarray(b.state[20 * offs[r]:20 * (offs[r] + L)].reshape(5, 1, L, 2, 2))
        oracle.step(x, oracle.make_cfg(1, L, 1, *b.couplings[r]), c["steps"], th)
        idx = sample_sites(x, L, 256, 10 + r)
        sites.append(offs[r] + idx)
        samples.append(x.reshape(5, -1, 2, 2)[:, idx])
    out["batch1d_steps"] = c["steps"]
    out["batch1d_sites"] = np.concatenate(sites)
    out["batch1d_samples"] = np.concatenate(samples, axis=1)

    c = W["batch2d"]
    b2 = c["w"]
    heights = b2.meta["heights"]
    sizes = b2.lengths * heights
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    sites, samples = [], []
    for r in range(len(heights)):
        nx, ny = int(b2.lengths[r]), int(heights[r])
        x = np.ascontiguousarray(b2.state[20 * offs[r]:20 * (offs[r] + nx * ny)].reshape(5, ny, nx, 2, 2))
        oracle.step(x, oracle.make_cfg(2, nx, ny, *b2.couplings[r]), c["steps"], th)
        idx = sample_sites(x, nx * ny, 1024, 20 + r)
        sites.append(offs[r] + idx)
        samples.append(x.reshape(5, -1, 2, 2)[:, idx])
    out["batch2d_steps"] = c["steps"]
    out["batch2d_sites"] = np.concatenate(sites)
    out["batch2d_samples"] = np.concatenate(samples, axis=1)

    c = W["adjoint"]
    w4 = c["w"]
    x0 = np.ascontiguousarray(w4.state)
    cot = inputs.adjoint_cotangent(x0.shape, c["cotangent_seed"])
    dg = oracle.vjp_run(x0, c["steps"], cot, oracle.make_cfg(2, w4.nx, w4.ny, *w4.g), th)
    idx = sample_sites(cot, w4.nx * w4.ny, 1024, 30)
    out["adjoint_steps"] = c["steps"]
    out["adjoint_sites"] = idx
    out["adjoint_cot_samples"] = cot.reshape(5, -1, 2, 2)[:, idx]
    out["adjoint_dg"] = np.asarray(dg)
    np.savez_compressed(os.path.join(HERE, "path_accuracy.npz"), **out)


if __name__ == "__main__":
    main()
