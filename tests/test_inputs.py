"""The seeded input generators against the recipes they state: shapes, the split a = b = eps psi / 2
of the boson field (Sec. VII.A), periodic kicks 2 pi n / L (Sec. IV.B), the unit background and
the winding of the Pade vortex dipoles (Table III, Sec. VI.A), the length and coupling
distributions of the batches, and determinism under the seed.  CPU only; the oracle pins check the
physics of the analytic states themselves."""
import numpy as np
import pytest

from paper_1907_12834_gb300 import inputs as I


def boson(w):
    return I.state_to_boson(w.state) / w.eps


def winding(phase, x0, x1, y0, y1):
    """Sum of the wrapped phase differences around the box [x0, x1] x [y0, y1] (counter-clockwise
    in (x, y)), over 2 pi."""
    path = ([(x, y0) for x in range(x0, x1)] + [(x1, y) for y in range(y0, y1)] +
            [(x, y1) for x in range(x1, x0, -1)] + [(x0, y) for y in range(y1, y0, -1)])
    path.append(path[0])
    d = np.array([phase[b[1], b[0]] - phase[a[1], a[0]] for a, b in zip(path[:-1], path[1:])])
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return d.sum() / (2 * np.pi)


def test_qubit_pair_split_and_shapes():
    w = I.config0()
    assert w.state.shape == (5, 1, 1024, 2, 2) and w.state.dtype == np.float64
    assert (w.ndim, w.nx, w.ny, w.steps, w.precision) == (1, 1024, 1, 2000, 64)
    np.testing.assert_array_equal(w.state[..., 0, :], w.state[..., 1, :])      # a == b
    psi = boson(w)
    # row 1 occupies m = +2 only; the soliton sits at the lattice centre with width 1 / (k eps)
    assert np.abs(psi[1:]).max() == 0.0
    j = int(np.argmax(np.abs(psi[0, 0])))
    assert abs(j - 512) <= 1
    x = 0.1 * (np.arange(1024) - 512)
    prof = np.abs(psi[0, 0])
    np.testing.assert_allclose(prof / prof.max(), 1.0 / np.cosh(x), rtol=0, atol=1e-12)


@pytest.mark.parametrize("couplings", [(1.0, -0.5, 0.2), (1.0, 0.8, -0.6)])
def test_config1_kicks_are_periodic_and_seeded(couplings):
    w = I.config1(couplings=couplings)
    assert (w.nx, w.ny, w.steps, w.g) == (16384, 1, 20000, couplings)
    n = w.meta["n_kick"]
    assert round(0.05 * 16384 / (2 * np.pi)) <= n <= round(0.3 * 16384 / (2 * np.pi))
    assert len(set(w.meta["rows"])) == 2 and set(w.meta["rows"]) <= {1, 2, 15}
    psi = boson(w)[:, 0, :]
    # the field continues smoothly across the periodic boundary: the step from site L - 1 to
    # site 0 is no larger than the steps inside the lattice (an aperiodic kick leaves a jump)
    inner = np.abs(np.diff(psi, axis=1)).max()
    assert np.abs(psi[:, 0] - psi[:, -1]).max() <= inner
    # the two solitons sit at L/4 and 3L/4 with equal and opposite momenta 2 pi n / L
    dens = (np.abs(psi) ** 2).sum(0)
    assert abs(int(np.argmax(dens[:8192])) - 4096) <= 2
    assert abs(8192 + int(np.argmax(dens[8192:])) - 12288) <= 2
    ph = np.unwrap(np.angle(psi[:, 4000:4200][np.abs(psi[:, 4096]).argmax()]))
    np.testing.assert_allclose(np.diff(ph), 2 * np.pi * n / 16384, atol=1e-9)
    again = I.config1(couplings=couplings)
    np.testing.assert_array_equal(w.state, again.state)


def test_config2_recipe_on_a_small_lattice():
    n, sep = 256, 64
    w = I.config2(n=n)
    assert w.state.shape == (5, n, n, 2, 2) and w.state.dtype == np.float32
    assert w.g == (1.0, 0.1, 1.0) and w.steps == 5000
    psi = boson(w)
    # variant a: only m = +2 and m = -2 occupied; the Pade profile rises to the unit background
    # from below (b1 > a1), as 1 - O(1 / r^2): within 2% at the corner of a 256^2 lattice
    assert np.abs(psi[1:4]).max() == 0.0
    far = np.abs(psi[0, :16, :16])
    assert 0.98 < far.min() and far.max() < 1.0
    # no site on a core (cores sit half a site off the lattice points)
    assert np.abs(psi[0]).min() > 0.0 and np.abs(psi[4]).min() > 0.0
    # m = +2: vortex (+1) at x1 = n/2 + 0.5 - sep/2, antivortex (-1) at x2; m = -2 counter-rotating
    cx, cy = n / 2 + 0.5, n / 2 + 0.5
    for lev, sign in ((0, +1), (4, -1)):
        ph = np.angle(psi[lev])
        for xc, wind in ((cx - sep / 2, +1), (cx + sep / 2, -1)):
            x0, y0 = int(xc) - 8, int(cy) - 8
            assert round(winding(ph, x0, x0 + 16, y0, y0 + 16)) == sign * wind
        # a loop around both cores encloses no net winding
        assert round(winding(ph, int(cx - sep), int(cx + sep), int(cy) - 16, int(cy) + 16)) == 0
    assert I.dipole_cores(n, n, sep) == [(0, cx - sep / 2, cy), (0, cx + sep / 2, cy),
                                         (4, cx - sep / 2, cy), (4, cx + sep / 2, cy)]


def test_config3_batch_distribution():
    w = I.config3()
    L = w.lengths
    assert len(L) == 256 and L.min() >= 2048 and L.max() <= 65536
    # log-uniform in [2048, 65536]: log2 L uniform in [11, 16]
    lg = np.log2(L)
    assert abs(lg.mean() - 13.5) < 0.3
    assert abs(np.quantile(lg, 0.25) - 12.25) < 0.4 and abs(np.quantile(lg, 0.75) - 14.75) < 0.4
    assert w.state.size == 20 * int(L.sum()) and w.state.dtype == np.float32
    np.testing.assert_array_equal(w.couplings[:, 0], 1.0)
    assert np.abs(w.couplings[:, 1:]).max() <= 1.0
    assert w.couplings[:, 1].min() < -0.8 and w.couplings[:, 1].max() > 0.8
    r = 17
    st = w.run_state(r)
    assert st.shape == (5, 1, int(L[r]), 2, 2)
    np.testing.assert_array_equal(st[..., 0, :], st[..., 1, :])


def test_batch2d_sizes_and_couplings():
    w = I.batch2d()
    nx, ny = w.lengths, w.meta["heights"]
    assert len(nx) == 128 and (nx % 32 == 0).all() and nx.min() >= 64 and nx.max() <= 512
    assert ny.min() >= 64 and ny.max() <= 512
    assert w.state.size == 20 * int((nx * ny).sum())
    g = w.couplings
    assert (g[:, 0] == 1.0).all()
    assert (0.05 <= g[:, 1]).all() and (g[:, 1] <= 0.5).all()
    assert (0.5 <= g[:, 2]).all() and (g[:, 2] <= 1.5).all()


def test_config4_is_the_config2_recipe_at_its_own_seed():
    w = I.config4(n=128, separation=32)
    ref = I.config2(seed=1911, n=128, separation=32)
    np.testing.assert_array_equal(w.state, ref.state)
    assert len(w.meta["cores"]) == 4


def test_perturbation_is_relative_and_seeded():
    x0 = I.config0().state
    p = I.perturbed(x0)
    rel = np.abs(p - x0)[x0 != 0] / np.abs(x0[x0 != 0])
    assert 1e-16 < np.median(rel) < 1e-13 and rel.max() < 1e-12
    np.testing.assert_array_equal(p, I.perturbed(x0))
