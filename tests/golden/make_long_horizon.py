"""Writes tests/golden/long_horizon_<workload>.npz: the FP64 oracle's trajectory of a long run,
the expected values of the long-horizon accuracy record.

Calls only the oracle (oracle/) and the seeded input generators (paper_1907_12834_gb300.inputs,
which hold none of the method's arithmetic).  For each workload the oracle runs the full step
count from the workload's initial state and, separately, from that state perturbed by a relative
1e-13 (x0 (1 + 1e-13 xi), xi seeded standard normal).  Every `every` steps it records:
  * the state at a sample of sites (the GPU runs are compared there): the sites of
    largest density at that step (3/4 of the sample; they carry most of the norm of a
    localised soliton field) and a seeded uniform draw of the others,
  * the relative L2 distance between the two oracle runs over the whole lattice (how much the
    dynamics itself amplifies a rounding-sized difference; the relative L2 error is the
    accuracy measure of Sec. VII.B's convergence study),
  * the qubit norm of the unperturbed run (exactly conserved by the algorithm).

  python tests/golden/make_long_horizon.py NAME [--threads N]      NAME in WORKLOADS
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1907_12834_gb300 import inputs  # noqa: E402

SAMPLE_SITES = {1: 256, 2: 1024}   # per dimension: a 1D soliton field is localised, a 2D
                                    # vortex field fills the lattice


workload = inputs.long_horizon_workload
WORKLOADS = inputs.LONG_HORIZON


def sample_sites(x, nsites, seed, count):
    """Indices (sorted) of the sample of `count` sites: the 3/4 count densest sites, then a
    seeded uniform draw among the rest."""
    dens = (x.reshape(5, nsites, 4) ** 2).sum(axis=(0, 2))
    ntop = (3 * count) // 4
    top = np.argsort(-dens, kind="stable")[:ntop]
    rest = np.setdiff1d(np.arange(nsites), top)
    rng = np.random.default_rng(seed)
    extra = rng.choice(rest, size=count - ntop, replace=False)
    return np.sort(np.concatenate([top, extra]))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=WORKLOADS)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    ndim, nx, ny, g, steps, every, x0 = workload(args.name)
    cfg = oracle.make_cfg(ndim, nx, ny, *g)
    n = nx * ny
    x = x0.copy()
    xp = inputs.perturbed(x0)

    def record(k):
        idx = sample_sites(x, n, 1907 + k, SAMPLE_SITES[ndim])
        checkpoints.append(k)
        sites.append(idx)
        samples.append(x.reshape(5, n, 2, 2)[:, idx])
        growth.append(rel_l2(xp, x))
        norms.append(float((x ** 2).sum()))

    checkpoints, sites, samples, growth, norms = [], [], [], [], []
    record(0)
    t0 = time.time()
    for k in range(every, steps + 1, every):
        oracle.step(x, cfg, every, args.threads)
        oracle.step(xp, cfg, every, args.threads)
        record(k)
        print("%s step %d: perturbed/unperturbed %.3e (%.0f s)" % (args.name, k, growth[-1], time.time() - t0),
              flush=True)
    np.savez_compressed(os.path.join(HERE, "long_horizon_%s.npz" % args.name), ndim=ndim, nx=nx, ny=ny,
                        g=np.asarray(g), steps=np.asarray(checkpoints), sites=np.asarray(sites),
                        samples=np.asarray(samples), oracle_growth=np.asarray(growth),
                        norm_qubit=np.asarray(norms), perturbation=inputs.PERTURBATION)


if __name__ == "__main__":
    main()
