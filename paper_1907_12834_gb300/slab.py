"""Slab decomposition of a 2D lattice along y (Sec. VII.C: the lattice split over several GPUs).

A lattice of nx x ny sites is cut along y into slabs of whole rows.  Each slab is an ordinary
library handle whose lattice holds the slab's rows plus HALO rows on each side, so its own
periodic wrap in y only ever reaches halo rows.  One QLGA step moves a site's dependency cone at
most 4 rows along y (the four kinetic blocks of the axis, Sec. VII.B), so when the halo rows hold
the neighbouring slabs' rows before every step, the slab's own rows come out exactly as in the
whole lattice.  The fifth halo row serves the forward difference of the energy at the slab's
last row.  Halo rows are stale after a step until the next exchange; a read-out needs a fresh
exchange too.

Two ways to exchange the halo rows:
  * exchange_local(slabs): all slabs in one process (one device, or devices with peer access),
    handle to handle with qlga_exchange_rows;
  * exchange_halos(slab, rank, world, dist): one slab per rank; the boundary rows are copied out
    with qlga_copy_rows, sent to the neighbouring ranks with torch.distributed point-to-point
    messages (NCCL for device tensors; through host memory for gloo) and copied into the halo.
The observables of the whole lattice are the sums over the slabs' own rows (one all-reduce of 14
doubles), turned into qlga_obs by qlga_obs_from_sums.
"""
from __future__ import annotations

import numpy as np

from . import qlga

HALO = 5   # rows on each side: 4 for a step's dependency cone along y, 1 for the energy pair


def partition_rows(ny: int, nslabs: int):
    """(y0, rows) of each slab: consecutive whole rows, sizes differing by at most one; every
    slab needs at least HALO rows (its halo rows come from the adjacent slabs only)."""
    if nslabs < 1:
        raise ValueError("nslabs must be >= 1")
    if ny < HALO * nslabs:
        raise ValueError("ny = %d is too small for %d slabs of at least %d rows" % (ny, nslabs, HALO))
    bounds = [(ny * k) // nslabs for k in range(nslabs + 1)]
    return [(bounds[k], bounds[k + 1] - bounds[k]) for k in range(nslabs)]


def halo_plan(rows: int):
    """Local row ranges of a slab with `rows` own rows held at offset HALO:
    send_down: its first HALO own rows, which the slab below keeps as its upper halo;
    send_up:   its last HALO own rows, which the slab above keeps as its lower halo;
    recv_down: the lower halo, filled from the slab below;  recv_up: the upper halo."""
    return {"send_down": (HALO, HALO), "send_up": (rows, HALO),
            "recv_down": (0, HALO), "recv_up": (HALO + rows, HALO)}


def extended_rows(state, y0: int, rows: int):
    """Rows y0 - HALO .. y0 + rows + HALO - 1 (periodic) of a whole-lattice state array of
    the library layout (5, ny, nx, 2, 2): a slab's initial state with its halo."""
    ny = state.shape[1]
    idx = [(y0 - HALO + k) % ny for k in range(rows + 2 * HALO)]
    return np.ascontiguousarray(state[:, idx])


def exchange_halos(slab, rank: int, world: int, dist=None, group=None):
    """Fill the halo rows of this rank's slab from the ranks above and below (periodic in y).

    `slab` provides rows_out(y0, n) -> tensor and rows_in(y0, tensor) over its local rows and
    `rows` (its own row count).  Messages: the last HALO own rows go up (tag 0), the first
    HALO own rows go down (tag 1); every rank posts its two sends, then its two receives, so the
    pairs match in order on backends without tags.  Device tensors go over the wire as they
    are when the backend is NCCL; with another backend they pass through host memory."""
    plan = halo_plan(slab.rows)
    up = slab.rows_out(*plan["send_up"])
    down = slab.rows_out(*plan["send_down"])
    if world == 1:
        slab.rows_in(plan["recv_down"][0], up)
        slab.rows_in(plan["recv_up"][0], down)
        return
    backend = dist.get_backend(group)
    via_host = backend != "nccl" and getattr(up, "is_cuda", False)
    send_up = up.cpu() if via_host else up
    send_down = down.cpu() if via_host else down
    recv_down = send_up.new_empty(send_up.shape)
    recv_up = send_down.new_empty(send_down.shape)
    above, below = (rank + 1) % world, (rank - 1) % world
    ops = [dist.P2POp(dist.isend, send_up, above, group, 0),
           dist.P2POp(dist.isend, send_down, below, group, 1),
           dist.P2POp(dist.irecv, recv_down, below, group, 0),
           dist.P2POp(dist.irecv, recv_up, above, group, 1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    if via_host:
        recv_down = recv_down.to(up.device)
        recv_up = recv_up.to(up.device)
    slab.rows_in(plan["recv_down"][0], recv_down)
    slab.rows_in(plan["recv_up"][0], recv_up)


def allreduce_sums(sums, dist=None, group=None, device=None):
    """Sum the 14 observable sums of every rank (one all-reduce of 14 doubles)."""
    if dist is None:
        return np.asarray(sums, dtype=np.float64)
    import torch
    t = torch.tensor(np.asarray(sums, dtype=np.float64), device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


class SlabLattice:
    """One slab of an nx x ny lattice on the current device: rows [y0, y0 + rows) held with
    HALO rows on each side in a library handle of nx x (rows + 2 HALO) sites (2D only)."""

    def __init__(self, nx, ny, nslabs, index, precision=64, g=(1.0, 0.0, 0.0), epsilon=0.1,
                 interleave=0, kinetic_variant=0, stream=None, device=None):
        self.nx, self.ny = int(nx), int(ny)
        self.y0, self.rows = partition_rows(self.ny, nslabs)[index]
        self.index, self.nslabs = index, nslabs
        self.lat = qlga.Lattice(2, nx, self.rows + 2 * HALO, precision=precision, g=g, epsilon=epsilon,
                                interleave=interleave, kinetic_variant=kinetic_variant, stream=stream,
                                device=device)
        self.steps = 0

    # row access for exchange_halos
    def rows_out(self, y0, n):
        return self.lat.copy_rows_out(y0, n)

    def rows_in(self, y0, rows):
        self.lat.copy_rows_in(y0, rows)

    def load_global(self, state):
        """Load this slab's rows (and halo) from a whole-lattice state array."""
        self.lat.load_state(extended_rows(state, self.y0, self.rows))
        self.steps = 0

    def step(self):
        """One step of the slab; the halo rows must have been exchanged since the last step."""
        self.lat.step(1)
        self.steps += 1

    def own_state(self):
        """The true state of the slab's own rows (halo rows exchanged first), numpy."""
        return self.lat.get_state()[:, HALO:HALO + self.rows]

    def own_sums(self, ref=None):
        """The 14 observable sums over the slab's own rows (halo rows exchanged first)."""
        return self.lat.observable_sums(HALO, HALO + self.rows, ref)

    def close(self):
        self.lat.close()


def exchange_local(slabs):
    """Fill every slab's halo rows from its neighbours (periodic in y) when all slabs live in
    this process: slabs[k] holds the k-th block of rows; rows move handle to handle."""
    n = len(slabs)
    for k, s in enumerate(slabs):
        below, above = slabs[(k - 1) % n], slabs[(k + 1) % n]
        qlga.qlga_exchange_rows(below.lat.handle, below.rows, s.lat.handle, 0, HALO)
        qlga.qlga_exchange_rows(above.lat.handle, HALO, s.lat.handle, HALO + s.rows, HALO)


def run_local(slabs, nsteps):
    """nsteps steps of all slabs of one process, exchanging halo rows before every step; the
    halo rows are exchanged once more at the end so that the slabs can be read out."""
    for _ in range(nsteps):
        exchange_local(slabs)
        for s in slabs:
            s.step()
    exchange_local(slabs)


def gather_local(slabs):
    """The whole lattice's true state from the slabs of one process (numpy, library layout)."""
    return np.concatenate([s.own_state() for s in slabs], axis=1)


def observables_local(slabs):
    """Observables of the whole lattice from the slabs of one process (halo rows fresh)."""
    sums = sum(s.own_sums() for s in slabs)
    return qlga.obs_to_dict(qlga.qlga_obs_from_sums(sums, slabs[0].steps))
