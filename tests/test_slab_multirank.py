"""Slab decomposition along y (Sec. VII.C) on CPU: the partition, the halo bookkeeping and the
point-to-point exchange, with gloo ranks on 127.0.0.1 and the FP64 oracle as the step engine.

Each rank holds its rows of a 2D lattice with HALO rows on each side and steps them with the
oracle on that extended lattice (periodic in y within it), exchanging halo rows with the ranks
above and below before every step through slab.exchange_halos.  The dependency cone of one step
is 4 rows along y, so the ranks' own rows must equal the whole-lattice oracle run bit for bit:
every site sees the same neighbour values and runs the same arithmetic.  The observables are
sums over the ranks' own rows, combined by one all-reduce (slab.allreduce_sums)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1907_12834_gb300 import inputs as I  # noqa: E402
from paper_1907_12834_gb300 import slab  # noqa: E402

G = (1.0, 0.8, -0.6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleSlab:
    """A slab as an FP64 array of the library layout, with HALO rows on each side."""

    def __init__(self, state, y0, rows, interleave):
        self.rows = rows
        self.nx = state.shape[2]
        self.ext = slab.extended_rows(state, y0, rows).astype(np.float64)
        self.cfg = oracle.make_cfg(2, self.nx, rows + 2 * slab.HALO, *G, interleave=interleave)

    def rows_out(self, y0, n):
        return torch.from_numpy(np.ascontiguousarray(self.ext[:, y0:y0 + n]).reshape(5, n, self.nx, 4))

    def rows_in(self, y0, t):
        n = int(t.shape[1])
        self.ext[:, y0:y0 + n] = t.numpy().reshape(5, n, self.nx, 2, 2)

    def step(self):
        oracle.step(self.ext, self.cfg, 1)

    def own(self):
        return self.ext[:, slab.HALO:slab.HALO + self.rows]


def _global_run(nx, ny, nsteps, interleave):
    rng = np.random.default_rng(1907 + nx + ny)
    st = I.random_state(rng, nx, ny, scale=0.08)
    ref = np.array(st, dtype=np.float64)       # a copy: the oracle steps in place
    oracle.step(ref, oracle.make_cfg(2, nx, ny, *G, interleave=interleave), nsteps)
    return st, ref


def _worker(rank, world, port, nx, ny, nsteps, interleave, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st, _ = _global_run(nx, ny, 0, interleave)
        y0, rows = slab.partition_rows(ny, world)[rank]
        s = OracleSlab(st, y0, rows, interleave)
        for _ in range(nsteps):
            slab.exchange_halos(s, rank, world, dist)
            s.step()
        parts = [None] * world
        dist.all_gather_object(parts, (y0, s.own().copy()))
        own = s.own()
        sums = np.zeros(14)
        sums[0] = float((own ** 2).sum())                                  # qubit norm
        sums[2:7] = (own ** 2).sum(axis=(1, 2, 3, 4))                      # populations
        total = slab.allreduce_sums(sums, dist, device="cpu")
        if rank == 0:
            out["parts"] = parts
            out["total"] = total
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nx,ny,nsteps,interleave", [(2, 16, 23, 6, 0), (3, 12, 17, 5, 0),
                                                           (2, 16, 20, 3, 1)])
def test_slabs_over_gloo_ranks_match_the_whole_lattice(world, nx, ny, nsteps, interleave):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), nx, ny, nsteps, interleave, out), nprocs=world,
                       start_method="spawn")
    _, ref = _global_run(nx, ny, nsteps, interleave)
    parts = sorted(out["parts"], key=lambda p: p[0])
    got = np.concatenate([p[1] for p in parts], axis=1)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)                   # same arithmetic on every site: bit for bit
    total = out["total"]
    assert total[0] == pytest.approx(float((ref ** 2).sum()), rel=1e-13)
    np.testing.assert_allclose(total[2:7], (ref ** 2).sum(axis=(1, 2, 3, 4)), rtol=1e-13)


def test_one_rank_exchanges_with_itself():
    nx, ny, nsteps = 12, 14, 4
    st, ref = _global_run(nx, ny, nsteps, 0)
    s = OracleSlab(st, 0, ny, 0)
    for _ in range(nsteps):
        slab.exchange_halos(s, 0, 1)
        s.step()
    assert np.array_equal(s.own(), ref)


def test_partition_and_halo_plan():
    assert slab.partition_rows(23, 2) == [(0, 11), (11, 12)]
    assert slab.partition_rows(4096, 4) == [(0, 1024), (1024, 1024), (2048, 1024), (3072, 1024)]
    parts = slab.partition_rows(37, 3)
    assert sum(r for _, r in parts) == 37 and all(r >= slab.HALO for _, r in parts)
    assert all(parts[k][0] + parts[k][1] == parts[k + 1][0] for k in range(2))
    with pytest.raises(ValueError):
        slab.partition_rows(9, 2)                      # fewer than HALO rows per slab
    with pytest.raises(ValueError):
        slab.partition_rows(10, 0)
    p = slab.halo_plan(11)
    H = slab.HALO
    assert p["send_down"] == (H, H) and p["send_up"] == (11, H)
    assert p["recv_down"] == (0, H) and p["recv_up"] == (H + 11, H)
    # the rows sent up are the receiver's lower halo: global rows y0 + rows - H .. y0 + rows - 1
    st = np.arange(5 * 23 * 4 * 4, dtype=np.float64).reshape(5, 23, 4, 2, 2)
    lo = slab.extended_rows(st, 0, 11)
    hi = slab.extended_rows(st, 11, 12)
    assert np.array_equal(lo[:, 11:11 + H], hi[:, 0:H])             # send_up -> recv_down
    assert np.array_equal(hi[:, H:2 * H], lo[:, H + 11:2 * H + 11])  # send_down -> recv_up
    assert np.array_equal(lo[:, 0:H], st[:, 23 - H:23])             # periodic wrap at y = 0
