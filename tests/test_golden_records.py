"""The stored oracle records under tests/golden/ (written by make_long_horizon.py and
make_path_accuracy.py, which call only the oracle) against the input recipes they were made from
and against what the algorithm conserves.  CPU only: no GPU and no oracle run here.

* The step-0 sample of every long-horizon record equals the workload's initial state at those
  sites, as the recipe in paper_1907_12834_gb300.inputs produces it today; a change to a recipe
  that would invalidate the record fails here.
* The qubit norm, conserved exactly by every QLGA step (unitary collide, stream and potential),
  holds to FP64 rounding: at most 2e-15 relative per step over the stored trajectories (the
  oracle's U from a Jacobi eigendecomposition is unitary to about 5e-16 per step).
* Sample sites are sorted, distinct and inside the lattice; the perturbed run starts 1e-13 away.
"""
import os

import numpy as np
import pytest

from paper_1907_12834_gb300 import inputs

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", inputs.LONG_HORIZON)
def test_long_horizon_record(name):
    path = os.path.join(GOLD, "long_horizon_%s.npz" % name)
    if not os.path.exists(path):
        pytest.skip("record not written")
    G = np.load(path)
    ndim, nx, ny, g, steps, every, x0 = inputs.long_horizon_workload(name)
    assert int(G["ndim"]) == ndim and int(G["nx"]) == nx and int(G["ny"]) == ny
    np.testing.assert_array_equal(G["g"], np.asarray(g))
    np.testing.assert_array_equal(G["steps"], np.arange(0, steps + 1, every))
    n = nx * ny
    for idx in G["sites"]:
        assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < n
    np.testing.assert_array_equal(G["samples"][0], x0.reshape(5, n, 2, 2)[:, G["sites"][0]])
    norms = G["norm_qubit"]
    assert norms[0] == pytest.approx(float((x0 ** 2).sum()), rel=1e-14)
    drift = np.abs(norms - norms[0]) / norms[0]
    assert np.all(drift <= 2e-15 * G["steps"] + 1e-15), drift.tolist()
    growth = G["oracle_growth"]
    assert growth[0] == pytest.approx(inputs.PERTURBATION, rel=0.05)
    assert np.all(np.isfinite(growth))


def test_path_accuracy_record():
    path = os.path.join(GOLD, "path_accuracy.npz")
    if not os.path.exists(path):
        pytest.skip("record not written")
    G = np.load(path)
    W = inputs.path_accuracy_workloads()
    w0 = W["config0"]["w"]
    x0 = np.asarray(w0.state, dtype=np.float64)
    xn = G["config0_state"]
    assert xn.shape == x0.shape
    assert float((xn ** 2).sum()) == pytest.approx(float((x0 ** 2).sum()), rel=1e-12)
    # config 0 is the stationary Table I row 1 soliton: the level populations stay put (only
    # m = +2 is occupied, so V is diagonal) -- the record's own physics check
    pop0 = (x0 ** 2).sum(axis=(1, 2, 3, 4))
    popn = (xn ** 2).sum(axis=(1, 2, 3, 4))
    np.testing.assert_allclose(popn, pop0, rtol=0, atol=1e-12 * pop0.sum())
    wi = W["interleaved"]["w"]
    assert G["interleaved_samples"].shape == (5, len(G["interleaved_sites"]), 2, 2)
    assert G["interleaved_sites"][-1] < wi.nx * wi.ny
    b = W["batch1d"]["w"]
    assert G["batch1d_sites"][-1] < int(b.lengths.sum())
    b2 = W["batch2d"]["w"]
    assert G["batch2d_sites"][-1] < int((b2.lengths * b2.meta["heights"]).sum())
    assert G["adjoint_dg"].shape == (3,) and np.all(np.isfinite(G["adjoint_dg"]))
