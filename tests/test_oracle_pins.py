"""The FP64 CPU oracle pinned to what the paper and the mathematics fix (no GPU needed)."""
import numpy as np
import pytest

import golden
import oracle
import pins
from paper_1907_12834_gb300 import inputs as I


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


# ---------------------------------------------------------------- the potential V(psi)

def test_table1_rows_are_eigenvectors_of_V(orc):
    """Sec. III.A / Table I: every real Thomas-Fermi row satisfies V(c) c = E c."""
    assert pins.pin_table1(orc) < 1e-13


def test_table1_transcriptions_agree():
    """The input generator's Table I and the golden transcription are the same table."""
    for E, g0, g1, g2 in pins.COUPLING_SETS:
        for row, c in golden.table1(E, g0, g1, g2).items():
            np.testing.assert_allclose(I.table1_coefficients(row, E, g0, g1, g2, c1=0.3, c2=0.2),
                                       c, rtol=0, atol=1e-15)


def test_table2_characteristics(orc):
    """Sec. III.B / Table II: |F_par|, |F_perp|, |A00| of the Table I rows."""
    assert pins.pin_table2(orc) < 1e-12


def test_V_is_hermitian_and_spin_parts_separate(orc):
    rng = np.random.default_rng(1)
    psi = rng.normal(size=5) + 1j * rng.normal(size=5)
    V = orc.potential_matrix(psi, 0.7, -0.3, 0.4)
    np.testing.assert_allclose(V, V.conj().T, atol=1e-15)
    # trace: 5 g0 rho + g1 tr(F.f) + g2/5 |s|^2 = 5 g0 rho + g2 rho / 5 (f traceless, |s| = |psi|)
    rho = float(np.vdot(psi, psi).real)
    assert abs(np.trace(V).real - (5 * 0.7 * rho + 0.4 * rho / 5)) < 1e-13


# ---------------------------------------------------------------- the exponential

def test_expm_matches_scipy_and_is_unitary(orc):
    assert pins.pin_expm(orc) < 1e-13


# ---------------------------------------------------------------- kinetic operator

@pytest.mark.parametrize("variant", [0, 1])
def test_kinetic_plane_wave_symbol(orc, variant):
    """Whole-lattice collide/stream sweeps equal the closed-form Fourier symbol on every
    plane wave of a 12-site ring and a 6 x 5 torus."""
    assert pins.pin_plane_wave_symbol(orc, variant) < 1e-13


@pytest.mark.parametrize("variant", [0, 1])
def test_kinetic_is_one_minus_i_p_squared(orc, variant):
    """Sec. VII.B: I'_1 I'_1 I'_2 I'_2 psi = psi - i p^2 psi + O(p^4) on the boson mode."""
    # the O(p^4) remainder divided by p^4 stays bounded (0.6 for K1, 1.4 for K2) as p -> 0
    assert pins.kinetic_phase_error(orc, variant) < 2.0


def test_kinetic_symbol_phase_and_leak():
    """The boson (a = b) mode gains phase -(k^2 - k^4/3) and leaks O(k^5) into a - b."""
    s = np.array([1, 1]) / np.sqrt(2)
    d = np.array([1, -1]) / np.sqrt(2)
    for k in (0.01, 0.05, 0.1):
        K = pins.kinetic_symbol(k)
        ph = np.angle(np.vdot(s, K @ s))
        assert abs(ph + (k ** 2 - k ** 4 / 3)) < 2 * k ** 6
        assert abs(np.vdot(d, K @ s)) < k ** 5


def test_kinetic_conserves_level_populations(orc):
    rng = np.random.default_rng(2)
    st = rng.normal(size=(5, 5, 7, 2, 2))
    cfg = oracle.make_cfg(2, 7, 5, 0, 0, 0)
    p0 = (st ** 2).sum(axis=(1, 2, 3, 4))
    orc.apply_kinetic(st, cfg)
    np.testing.assert_allclose((st ** 2).sum(axis=(1, 2, 3, 4)), p0, rtol=1e-14)


# ---------------------------------------------------------------- the whole step

@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("interleave", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
def test_step_matches_dense_operator_product(orc, ndim, interleave, variant):
    """Brute force: the step equals the product of dense C, S, U matrices (L=4, 3x3)."""
    assert pins.pin_dense_step(orc, ndim, interleave, variant) < 1e-13


@pytest.mark.parametrize("interleave", [0, 1])
def test_uniform_thomas_fermi_state_gains_exact_phase(orc, interleave):
    assert pins.pin_tf_phase(orc, interleave) < 1e-13


@pytest.mark.parametrize("ndim", [1, 2])
def test_step_is_unitary(orc, ndim):
    assert pins.pin_norm(orc, ndim) < 1e-13


# ---------------------------------------------------------------- observables

def test_observables_closed_forms(orc):
    """Uniform Thomas-Fermi rows: energy density = E rho / 2 (c^dagger V(c) c = E rho with
    g0 rho^2 + g1 |F|^2 + g2/5 |psi^T J psi|^2 = c^dagger V c); populations |c_m|^2 / 2 per
    qubit; singlet sum of row 5 = N c_0^2 / sqrt(5); overlap with itself = boson norm."""
    E, g0, g1, g2 = 0.02, 1.0, 0.1, 1.0
    nx, ny = 4, 3
    N = nx * ny
    for row, c in golden.table1(E, g0, g1, g2, c1=0.03, c2=0.02).items():
        c = np.asarray(c)
        st = np.zeros((5, ny, nx, 2, 2))
        st[..., 0, 0] = st[..., 1, 0] = (c / 2)[:, None, None]
        cfg = oracle.make_cfg(2, nx, ny, g0, g1, g2)
        o = orc.observables(st, cfg, ref=st)
        rho = float((c ** 2).sum())
        assert abs(o["energy"] - N * E * rho / 2) < 1e-15
        np.testing.assert_allclose(o["pop"], N * c ** 2 / 2, atol=1e-16)
        assert abs(o["magnetisation"] - N * np.dot([2, 1, 0, -1, -2], c ** 2) / 2) < 1e-16
        assert abs(o["norm_boson"] - N * rho) < 1e-15
        assert abs(o["overlap_re"] - N * rho) < 1e-15 and abs(o["overlap_im"]) < 1e-15
        if row == 5:
            assert abs(o["singlet_re"] - N * c[2] ** 2 / np.sqrt(5)) < 1e-15
            assert abs(o["singlet_fraction"] - 1.0) < 1e-12


def test_observables_pin(orc):
    """The closed forms of pins.pin_observables (also used by the mutation tests)."""
    assert pins.pin_observables(orc) < 1e-12


def test_observables_plane_wave_gradient(orc):
    """Forward-difference kinetic energy of A e^{i k x}: 2 |A|^2 (1 - cos k) per site."""
    nx, ny = 16, 4
    k = 2 * np.pi * 3 / nx
    A = 0.3 + 0.1j
    st = np.zeros((5, ny, nx, 2, 2))
    w = A * np.exp(1j * k * np.arange(nx)) / 2
    st[1, :, :, 0, 0] = st[1, :, :, 1, 0] = w.real
    st[1, :, :, 0, 1] = st[1, :, :, 1, 1] = w.imag
    o = orc.observables(st, oracle.make_cfg(2, nx, ny, 0, 0, 0))
    assert abs(o["energy"] - nx * ny * 2 * abs(A) ** 2 * (1 - np.cos(k))) < 1e-14


# ---------------------------------------------------------------- physics of the paper

def _centroid(st, L):
    rho = (I.state_to_boson(st).__abs__() ** 2).sum(axis=(0, 1))
    ang = 2 * np.pi * np.arange(L) / L
    z = (rho * np.exp(1j * ang)).sum()
    return (np.angle(z) % (2 * np.pi)) * L / (2 * np.pi)


def test_bright_soliton_stationary_and_phase_rate(orc):
    """Sec. IV.A: the row-1 bright soliton stays put.  On the lattice its density settles to a
    bounded O(eps^2) adjustment (second-order convergence at fixed physical time), and its
    phase turns at -E = k^2 per unit physical time, k^2 eps^2 per step (Sec. III.C,
    Sec. VII.A scaling)."""
    T = 2.0
    err = {}
    for eps in (0.1, 0.05):
        L = int(round(102.4 / eps))
        w = I.config0(row=1, L=L, eps=eps)
        cfg = oracle.make_cfg(1, L, 1, *w.g)
        st = w.state.copy()
        psi0 = I.state_to_boson(st)
        n = int(round(T / eps ** 2))
        orc.step(st, cfg, n)
        psi = I.state_to_boson(st)
        err[eps] = np.abs(np.abs(psi) ** 2 - np.abs(psi0) ** 2).sum() / (np.abs(psi0) ** 2).sum()
        ph = np.angle(np.vdot(psi0, psi))
        assert abs(ph - n * eps ** 2) < 0.02 * n * eps ** 2
    assert err[0.1] < 0.02
    assert 3.0 < err[0.1] / err[0.05] < 5.0          # O(eps^2)


def test_magnetisation_exact_for_single_level_state(orc):
    """Row 1 occupies m = +2 only, so V stays diagonal and every population is conserved."""
    w = I.config0(row=1, L=256)
    cfg = oracle.make_cfg(1, w.nx, 1, *w.g)
    st = w.state.copy()
    o0 = orc.observables(st, cfg)
    orc.step(st, cfg, 50)
    o1 = orc.observables(st, cfg)
    assert abs(o1["magnetisation"] - o0["magnetisation"]) < 1e-12 * o0["norm_qubit"]
    np.testing.assert_allclose(o1["pop"], o0["pop"], atol=1e-12 * o0["norm_qubit"])


def test_kicked_soliton_moves_at_2p_and_obeys_dispersion(orc):
    """Sec. III.C: a bright soliton kicked by e^{ipx} moves at 2p (m = 1/2) and has energy
    E = p^2 - k^2 (Eq. dispersion), measured with the discrete energy of Sec. IV.B."""
    L, eps, nk = 1024, 0.1, 8
    j = np.arange(L)
    p_lat = 2 * np.pi * nk / L
    psi = I.bright_soliton(eps * (j - L / 2), 1, I.CONFIG0_G) * np.exp(1j * p_lat * j)[None, :]
    st = I.boson_to_state(psi, eps)
    cfg = oracle.make_cfg(1, L, 1, *I.CONFIG0_G)
    x0 = _centroid(st, L)
    orc.step(st, cfg, 20)
    prev = st.copy()
    orc.step(st, cfg, 1)
    o = orc.observables(st, cfg, ref=prev)
    E_lat = -np.angle(complex(o["overlap_re"], -o["overlap_im"]))   # -arg <psi(t-1)|psi(t)>
    p = p_lat / eps
    assert abs(E_lat / eps ** 2 - (p ** 2 - 1.0)) < 0.02
    n = 100
    orc.step(st, cfg, n - 21)
    dx = _centroid(st, L) - x0
    assert abs(dx - 2 * p_lat * n) < 0.01 * 2 * p_lat * n


def _dip_centroid(st, L):
    """Position (sites) of the two density dips of a periodic dark pair, which sit half a lattice
    apart: the circular centroid of the density deficit at period L/2."""
    rho = (np.abs(I.state_to_boson(st)) ** 2).sum(axis=(0, 1))
    z = ((rho.max() - rho) * np.exp(4j * np.pi * np.arange(L) / L)).sum()
    return (np.angle(z) % (2 * np.pi)) * L / (4 * np.pi)


@pytest.mark.parametrize("nk", [0, 8])
def test_dark_soliton_pair_dispersion_and_velocity(orc, nk):
    """Dark solitons (Sec. III.C, Eq. darkdispersion): a kink c k tanh(k x) kicked by e^{ipx} has
    E = p^2 + 2k^2 and moves at 2p.  On the periodic lattice the paper's product of two kinks
    (Sec. IV.A, dark solitons) with L/2 = 51 physical units between them is an eigenstate up to
    e^{-2 k L/4} tails; row 1 at E = 2 (k = 1) with the couplings (1, 0.1, 1) that make it real.
    The energy is the discrete one of Sec. IV.B."""
    L, eps, g = 1024, 0.1, (1.0, 0.1, 1.0)
    j = np.arange(L)
    p_lat = 2 * np.pi * nk / L
    psi = I.dark_soliton_pair(eps * j, eps * L, 1, g) * np.exp(1j * p_lat * j)[None, :]
    st = np.ascontiguousarray(I.boson_to_state(psi, eps))
    cfg = oracle.make_cfg(1, L, 1, *g)
    x0 = _dip_centroid(st, L)
    orc.step(st, cfg, 20)
    prev = st.copy()
    orc.step(st, cfg, 1)
    o = orc.observables(st, cfg, ref=prev)
    E_lat = -np.angle(complex(o["overlap_re"], -o["overlap_im"]))   # -arg <psi(t-1)|psi(t)>
    p = p_lat / eps
    assert abs(E_lat / eps ** 2 - (p ** 2 + 2.0)) < 0.01
    n = 100
    orc.step(st, cfg, n - 21)
    dx = _dip_centroid(st, L) - x0
    assert abs(dx - 2 * p_lat * n) < 0.02 * 2 * p_lat * n + 0.05


def test_fields(orc):
    """Per-site F_par, F_perp, |A00|, colour map and vorticity (Sec. III.B, VI.B)."""
    assert pins.pin_fields(orc) < 1e-12


def test_pade_table3_solves_gp_to_order_r7():
    """Table III: the Pade vortex leaves a residual O(r^7) in the single-level GP equation
    E f = -(f'' + f'/r - f/r^2) + g f^3 (g = g0 + 4 g1, g0 + g1, g0 + g2/5 for |mf| = 2, 1, 0)."""
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    E, g0, g1, g2 = 1.0, 1.0, 0.1, 1.0
    tab = golden.table3(E, g0, g1, g2)
    for mf, geff in ((2, g0 + 4 * g1), (1, g0 + g1), (0, g0 + g2 / 5)):
        a1, b1, a2 = I.pade_coefficients(mf, E, g0, g1, g2)
        assert any(np.allclose((a1, b1, a2), t, rtol=1e-12) for t in tab[mf])
        A1, B1, A2 = (sp.Rational(str(v)) for v in (a1, b1, a2))
        f = sp.sqrt((A2 * r ** 4 + A1 * r ** 2) / (A2 * r ** 4 + B1 * r ** 2 + 1))
        res = -(sp.diff(f, r, 2) + sp.diff(f, r) / r - f / r ** 2) + geff * f ** 3 - E * f
        ser = sp.series(res, r, 0, 7).removeO()
        for pw in (1, 3, 5):
            coef = float(ser.coeff(r, pw))
            assert abs(coef) < 1e-9, (mf, pw, coef)
