"""Slab decomposition along y (Sec. VII.C) through the library: a 2D lattice cut into slabs, each
an ordinary handle with HALO rows on each side, halo rows exchanged before every step.

In one process the rows move handle to handle (qlga_exchange_rows); across processes they are
copied out and in (qlga_copy_rows) and sent between gloo ranks through host memory -- here two
ranks on the one GPU, which run independent kernels and meet only on the host.  The slabs' own
rows are compared element by element with the FP64 oracle run of the whole lattice (1e-11 FP64,
1e-5 FP32), and the observables from the per-slab sums with the oracle's."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1907_12834_gb300 import inputs as I  # noqa: E402
from paper_1907_12834_gb300 import qlga, slab  # noqa: E402

G = (1.0, 0.8, -0.6)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def oracle_run(st, nx, ny, nsteps, interleave=0, variant=0):
    ref = np.array(st, dtype=np.float64)
    cfg = oracle.make_cfg(2, nx, ny, *G, interleave=interleave, kinetic_variant=variant)
    oracle.step(ref, cfg, nsteps)
    return ref, cfg


@pytest.mark.parametrize("precision,nx,ny,nslabs,nsteps,interleave,variant", [
    (64, 64, 40, 2, 12, 0, 0),      # fused FP64 shapes
    (64, 40, 37, 3, 9, 0, 1),       # two-pass FP64, uneven slabs, second collide reading
    (32, 64, 48, 2, 15, 0, 0),      # fused FP32
    (32, 96, 30, 3, 8, 0, 1),
    (32, 40, 26, 2, 10, 0, 0),      # two-pass FP32 (nx not a multiple of 32)
    (64, 32, 24, 2, 6, 1, 0),       # interleaved step
    (32, 64, 12, 1, 7, 0, 0),       # one slab exchanging with itself
])
def test_slabs_in_one_process_match_the_oracle(precision, nx, ny, nslabs, nsteps, interleave, variant):
    rng = np.random.default_rng(nx * ny + nslabs)
    st = I.random_state(rng, nx, ny, scale=0.06)
    if precision == 32:
        st = st.astype(np.float32)
    slabs = [slab.SlabLattice(nx, ny, nslabs, k, precision=precision, g=G, interleave=interleave,
                              kinetic_variant=variant) for k in range(nslabs)]
    try:
        for s in slabs:
            s.load_global(st)
        slab.run_local(slabs, nsteps)
        got = slab.gather_local(slabs)
        obs = slab.observables_local(slabs)
    finally:
        for s in slabs:
            s.close()
    ref, cfg = oracle_run(st, nx, ny, nsteps, interleave, variant)
    assert rel_l2(got, ref) <= (1e-11 if precision == 64 else 1e-5)
    want = oracle.observables(ref, cfg)
    tol = 1e-12 if precision == 64 else 2e-6
    scale = want["norm_qubit"]
    for k in ("norm_qubit", "norm_boson", "magnetisation", "energy", "singlet_re", "singlet_im"):
        assert abs(obs[k] - want[k]) <= tol * max(scale, abs(want[k])), (k, obs[k], want[k])
    np.testing.assert_allclose(obs["pop"], want["pop"], rtol=0, atol=tol * scale)
    assert obs["step"] == nsteps


def test_slab_sums_add_up_to_the_whole_lattice():
    nx, ny = 64, 30
    rng = np.random.default_rng(5)
    st = I.random_state(rng, nx, ny, scale=0.06)
    with qlga.Lattice(2, nx, ny, precision=64, g=G) as lat:
        lat.load_state(st)
        lat.step(4)
        whole = lat.observable_sums()
        parts = lat.observable_sums(0, 11) + lat.observable_sums(11, 30)
        obs = lat.observables()
    np.testing.assert_allclose(parts, whole, rtol=1e-13, atol=1e-15 * abs(whole).max())
    o2 = qlga.obs_to_dict(qlga.qlga_obs_from_sums(whole, 4))
    for k in ("norm_qubit", "energy", "singlet_fraction", "magnetisation"):
        assert o2[k] == pytest.approx(obs[k], rel=1e-13, abs=1e-15)


def test_row_copies_reject_bad_arguments():
    with qlga.Lattice(2, 64, 16, precision=32, g=G) as a, qlga.Lattice(2, 32, 16, precision=32, g=G) as b:
        buf = torch.empty((5, 4, 64, 4), dtype=torch.float32, device="cuda")
        with pytest.raises(qlga.QlgaError) as e:
            qlga.qlga_copy_rows(a.handle, 14, 4, buf.data_ptr(), qlga.QLGA_ROWS_OUT)   # past ny
        assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
        with pytest.raises(qlga.QlgaError) as e:
            qlga.qlga_copy_rows(a.handle, 0, 4, buf.data_ptr(), 7)
        assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
        with pytest.raises(qlga.QlgaError) as e:
            qlga.qlga_exchange_rows(a.handle, 0, b.handle, 0, 4)                      # nx differs
        assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
        with pytest.raises(qlga.QlgaError) as e:
            qlga.qlga_exchange_rows(a.handle, 0, a.handle, 2, 4)                      # overlapping
        assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
        with pytest.raises(qlga.QlgaError) as e:
            qlga.qlga_observable_sums(a.handle, 5, 5)
        assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
        # a copy out and back in leaves the state unchanged
        st = I.random_state(np.random.default_rng(1), 64, 16, scale=0.05).astype(np.float32)
        a.load_state(st)
        rows = a.copy_rows_out(3, 4)
        a.copy_rows_in(3, rows)
        assert np.array_equal(a.get_state(), st)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nx, ny, nsteps, precision, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        rng = np.random.default_rng(nx + ny)
        st = I.random_state(rng, nx, ny, scale=0.06)
        if precision == 32:
            st = st.astype(np.float32)
        s = slab.SlabLattice(nx, ny, world, rank, precision=precision, g=G)
        s.load_global(st)
        for _ in range(nsteps):
            slab.exchange_halos(s, rank, world, dist)
            s.step()
        slab.exchange_halos(s, rank, world, dist)
        parts = [None] * world
        dist.all_gather_object(parts, (s.y0, s.own_state()))
        total = slab.allreduce_sums(s.own_sums(), dist, device="cpu")
        s.close()
        if rank == 0:
            out["parts"] = parts
            out["total"] = total
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("precision", [64, 32])
def test_slab_ranks_over_gloo_on_one_gpu(precision):
    import torch.multiprocessing as mp
    world, nx, ny, nsteps = 2, 64, 34, 8
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), nx, ny, nsteps, precision, out), nprocs=world,
                       start_method="spawn")
    rng = np.random.default_rng(nx + ny)
    st = I.random_state(rng, nx, ny, scale=0.06)
    if precision == 32:
        st = st.astype(np.float32)
    ref, cfg = oracle_run(st, nx, ny, nsteps)
    parts = sorted(out["parts"], key=lambda p: p[0])
    got = np.concatenate([p[1] for p in parts], axis=1)
    assert rel_l2(got, ref) <= (1e-11 if precision == 64 else 1e-5)
    obs = qlga.obs_to_dict(qlga.qlga_obs_from_sums(out["total"], nsteps))
    want = oracle.observables(ref, cfg)
    tol = 1e-12 if precision == 64 else 2e-6
    assert abs(obs["energy"] - want["energy"]) <= tol * max(want["norm_qubit"], abs(want["energy"]))
    assert abs(obs["norm_qubit"] - want["norm_qubit"]) <= tol * want["norm_qubit"]
