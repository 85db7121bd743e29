"""Batches of lattices (uneven sizes, per-run couplings; 1D runs and 2D runs) against the
oracle, run by run."""
import numpy as np
import pytest

import oracle
from paper_1907_12834_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1907_12834_gb300 import qlga  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def split(state, lengths):
    out, o = [], 0
    for L in lengths:
        out.append(np.asarray(state[o:o + 20 * L]).reshape(5, 1, L, 2, 2))
        o += 20 * L
    return out


def oracle_runs(state, lengths, couplings, nsteps, variant=0):
    res = []
    for st, L, g in zip(split(state, lengths), lengths, couplings):
        r = np.ascontiguousarray(st, dtype=np.float64).copy()
        oracle.step(r, oracle.make_cfg(1, int(L), 1, *g, kinetic_variant=variant), nsteps)
        res.append(r)
    return res


LENGTHS = [8, 37, 64, 128, 129, 255, 1000, 2048, 3001]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("variant", [0, 1])
def test_ragged_batch_matches_oracle_per_run(precision, use_graph, variant):
    rng = np.random.default_rng(53 + precision + variant)
    couplings = np.column_stack([np.ones(len(LENGTHS)), rng.uniform(-1, 1, len(LENGTHS)),
                                 rng.uniform(-1, 1, len(LENGTHS))])
    state = np.concatenate([I.random_state(rng, L, scale=0.05).ravel() for L in LENGTHS])
    state = state.astype(np.float32 if precision == 32 else np.float64)
    b = qlga.Batch1D(LENGTHS, couplings, precision=precision, kinetic_variant=variant,
                     use_graph=use_graph)
    b.load_state(state)
    n = 21                                              # odd: graph pairs plus a single step
    b.step(n)
    got = split(b.get_state(), LENGTHS)
    info = b.info()
    b.close()
    ref = oracle_runs(state, LENGTHS, couplings, n, variant)
    tol = 1e-11 if precision == 64 else 2e-5
    for gr, rr in zip(got, ref):
        assert rel_l2(gr, rr) <= tol
    assert info["tile_width"] in (32, 64, 128, 256, 120, 248) and info["sites_per_thread"] in (1, 2, 4)
    assert info["steps_per_launch"] in ((1, 2) if precision == 32 else (1,))
    assert (info["graph_steps"] > 0) == use_graph


# every launch shape of the tiled kernel, forced: one step per launch, and two (temporal blocking:
# the tile plus an 8-site halo staged once; FP32); 13 steps = replays plus a single step; runs
# shorter than a tile and its halo wrap several times
SHAPES_1 = [(32, 1), (64, 1), (128, 1), (256, 1), (64, 2), (128, 2), (64, 4)]
SHAPES_2 = [(64, 4), (128, 2), (64, 2), (256, 1)]


@pytest.mark.parametrize("shape", [s + (1,) for s in SHAPES_1] + [s + (2,) for s in SHAPES_2])
@pytest.mark.parametrize("use_graph", [True, False])
def test_forced_shapes_match_oracle_per_run(shape, use_graph):
    rng = np.random.default_rng(83)
    couplings = np.column_stack([np.ones(len(LENGTHS)), rng.uniform(-1, 1, len(LENGTHS)),
                                 rng.uniform(-1, 1, len(LENGTHS))])
    state = np.concatenate([I.random_state(rng, L, scale=0.05).ravel() for L in LENGTHS]).astype(np.float32)
    b = qlga.Batch(LENGTHS, couplings, precision=32, use_graph=use_graph)
    b.set_shape(*shape)
    b.load_state(state)
    n = 13
    b.step(n)
    got = split(b.get_state(), LENGTHS)
    info = b.info()
    b.close()
    ref = oracle_runs(state, LENGTHS, couplings, n)
    for gr, rr, L in zip(got, ref, LENGTHS):
        assert rel_l2(gr, rr) <= 2e-5, L
    assert info["steps_per_launch"] == shape[2]
    assert info["sites_per_thread"] == shape[1]
    assert info["tile_width"] == shape[0] * shape[1] - 8 * (shape[2] - 1)


@pytest.mark.parametrize("shape", [s + (1,) for s in SHAPES_1])
def test_forced_shapes_fp64(shape):
    rng = np.random.default_rng(89)
    couplings = np.column_stack([np.ones(len(LENGTHS)), rng.uniform(-1, 1, len(LENGTHS)),
                                 rng.uniform(-1, 1, len(LENGTHS))])
    state = np.concatenate([I.random_state(rng, L, scale=0.05).ravel() for L in LENGTHS])
    b = qlga.Batch(LENGTHS, couplings, precision=64)
    b.set_shape(*shape)
    b.load_state(state)
    b.step(9)
    got = split(b.get_state(), LENGTHS)
    b.close()
    for gr, rr in zip(got, oracle_runs(state, LENGTHS, couplings, 9)):
        assert rel_l2(gr, rr) <= 1e-11


def test_shape_errors():
    g = [[1.0, 0.1, 0.2]] * 2
    b = qlga.Batch([64, 100], g, precision=64)
    for args, status in (((64, 4, 2), qlga.QLGA_ERR_UNSUPPORTED), ((63, 1, 1), qlga.QLGA_ERR_INVALID_ARG),
                         ((64, 4, 3), qlga.QLGA_ERR_INVALID_ARG)):
        with pytest.raises(qlga.QlgaError) as e:
            b.set_shape(*args)
        assert e.value.status == status
    b.close()
    b = qlga.Batch([64, 100], g, precision=32, heights=[16, 1])       # a 2D run: one step per launch
    with pytest.raises(qlga.QlgaError) as e:
        b.set_shape(64, 4, 2)
    assert e.value.status == qlga.QLGA_ERR_UNSUPPORTED
    b.set_shape(64, 4, 1)
    b.set_shape()
    b.close()


def test_batch_observables_per_run():
    rng = np.random.default_rng(61)
    couplings = np.column_stack([np.ones(len(LENGTHS)), rng.uniform(-1, 1, len(LENGTHS)),
                                 rng.uniform(-1, 1, len(LENGTHS))])
    state = np.concatenate([I.random_state(rng, L, scale=0.05).ravel() for L in LENGTHS])
    b = qlga.Batch1D(LENGTHS, couplings, precision=64)
    b.load_state(state)
    b.step(4)
    obs = b.observables()
    cur = split(b.get_state(), LENGTHS)
    b.close()
    for o, st, L, g in zip(obs, cur, LENGTHS, couplings):
        w = oracle.observables(np.ascontiguousarray(st), oracle.make_cfg(1, L, 1, *g))
        for k in ("norm_qubit", "norm_boson", "magnetisation", "energy", "singlet_re", "singlet_im"):
            assert abs(o[k] - w[k]) <= 1e-12 * w["norm_qubit"], k
        np.testing.assert_allclose(o["pop"], w["pop"], rtol=0, atol=1e-12 * w["norm_qubit"])


def test_config3_full_batch_sampled_runs():
    """The 256-run batch (L log-uniform in [2048, 65536], per-run couplings) in FP32, 6 steps;
    eight runs checked against the oracle, and every run's qubit norm against its start."""
    w = I.config3()
    b = qlga.Batch1D(w.lengths, w.couplings, precision=32)
    b.load_state(w.state)
    o0 = b.observables()
    b.step(6)
    got = b.get_state()
    o1 = b.observables()
    b.close()
    runs = split(got, w.lengths)
    for r in (0, 17, 64, 100, 128, 200, 254, 255):
        ref = np.ascontiguousarray(w.run_state(r), dtype=np.float64).copy()
        oracle.step(ref, oracle.make_cfg(1, int(w.lengths[r]), 1, *w.couplings[r]), 6)
        assert rel_l2(runs[r], ref) <= 2e-5, r
    for a, c in zip(o0, o1):
        assert abs(c["norm_qubit"] - a["norm_qubit"]) <= 1e-5 * a["norm_qubit"]


# (nx, ny): 1D runs have ny = 1; 2D runs need nx a multiple of 32 (ragged row chunks, a single
# strip whose halo wraps onto itself at nx = 32)
SHAPES = [(100, 1), (64, 40), (37, 1), (96, 33), (32, 17), (128, 64), (8, 1)]


def split_shapes(state, shapes):
    out, o = [], 0
    for nx, ny in shapes:
        out.append(np.asarray(state[o:o + 20 * nx * ny]).reshape(5, ny, nx, 2, 2))
        o += 20 * nx * ny
    return out


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("variant", [0, 1])
def test_mixed_1d_2d_batch_matches_oracle_per_run(use_graph, variant):
    rng = np.random.default_rng(71 + variant)
    n_runs = len(SHAPES)
    couplings = np.column_stack([np.ones(n_runs), rng.uniform(-1, 1, n_runs), rng.uniform(-1, 1, n_runs)])
    state = np.concatenate([I.random_state(rng, nx, ny, scale=0.05).ravel() for nx, ny in SHAPES])
    state = state.astype(np.float32)
    lengths = [nx for nx, _ in SHAPES]
    heights = [ny for _, ny in SHAPES]
    b = qlga.Batch(lengths, couplings, precision=32, kinetic_variant=variant, use_graph=use_graph,
                   heights=heights)
    b.load_state(state)
    n = 13
    b.step(n)
    got = split_shapes(b.get_state(), SHAPES)
    obs = b.observables()
    b.close()
    for st, (nx, ny), g, gr, ob in zip(split_shapes(state, SHAPES), SHAPES, couplings, got, obs):
        ndim = 1 if ny == 1 else 2
        cfg = oracle.make_cfg(ndim, nx, ny, *g, kinetic_variant=variant)
        ref = np.ascontiguousarray(st, dtype=np.float64).copy()
        oracle.step(ref, cfg, n)
        assert rel_l2(gr, ref) <= 2e-5, (nx, ny)
        ro = oracle.observables(ref, cfg)
        assert abs(ob["energy"] - ro["energy"]) <= 1e-5 * abs(ro["energy"]), (nx, ny)
        assert abs(ob["norm_qubit"] - ro["norm_qubit"]) <= 1e-6 * ro["norm_qubit"]


def test_2d_batch_rejects_unsupported_runs():
    with pytest.raises(qlga.QlgaError) as e:
        qlga.Batch([64, 100], [[1, 0.1, 0.2]] * 2, precision=64, heights=[16, 1])
    assert e.value.status == qlga.QLGA_ERR_UNSUPPORTED
    with pytest.raises(qlga.QlgaError) as e:
        qlga.Batch([40], [[1, 0.1, 0.2]], precision=32, heights=[16])
    assert e.value.status == qlga.QLGA_ERR_INVALID_ARG
