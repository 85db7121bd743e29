"""Pins of the CPU oracle: checks against what the paper and the mathematics fix.

Each function takes an ``oracle.Oracle`` and returns the largest deviation it finds, so the
same check serves the pin tests (deviation below tolerance) and the mutation tests (a
planted mistake in a copy of the oracle source pushes it above).
"""
import numpy as np
import scipy.linalg as sl

import oracle
import golden

# (E, g0, g1, g2) sets; the last one is the bright-soliton case of the 1D configurations
COUPLING_SETS = [(1.0, 1.0, 0.1, 1.0), (2.0, 1.3, 0.4, 0.7), (1.0, 1.0, 0.3, -0.5),
                 (-2.0, 1.0, -0.5, 0.2)]

C_K1 = 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]])
C_K2 = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]])


def collide_pair(variant):
    """(first, second) collide of a kinetic block: K1 = (C, C), K2 = (C, C^dagger)."""
    if variant == 0:
        return C_K1, C_K1
    return C_K2, C_K2.conj().T


# ----------------------------------------------------------------- potential (Table I / II)

def pin_table1(orc):
    """max |V(c) c - E c| over every real Table I row and coupling set (Sec. III.A)."""
    worst, count = 0.0, 0
    for E, g0, g1, g2 in COUPLING_SETS:
        for row, c in golden.table1(E, g0, g1, g2).items():
            c = np.asarray(c, dtype=complex)
            V = orc.potential_matrix(c, g0, g1, g2)
            worst = max(worst, float(np.abs(V @ c - E * c).max()) / max(1.0, abs(E)))
            count += 1
    assert count >= 40
    return worst


def pin_table2(orc):
    """max deviation from Table II (Sec. III.B): F_par and F_perp read off V(c) at couplings
    (0, 1, 0), where V = F.f, and |A00| from the oracle's singlet sum on a one-site lattice.
    Entries flagged as misprints are skipped."""
    worst = 0.0
    for E, g0, g1, g2 in COUPLING_SETS[:3]:
        rows1 = golden.table1(E, g0, g1, g2)
        for row, ((fpar, fperp, a00), flags) in golden.table2(E, g0, g1, g2).items():
            if row not in rows1:
                continue
            c = np.asarray(rows1[row], dtype=complex)
            V = orc.potential_matrix(c, 0.0, 1.0, 0.0)
            worst = max(worst, abs(abs(V[0, 0].real / 2.0) - fpar))     # f_z[+2,+2] = 2
            if "perp-misprint" not in flags:
                worst = max(worst, abs(abs(V[1, 0]) - fperp))          # c_0 = 1: V[1,0] = F_+
            cfg = oracle.make_cfg(1, 1, 1, g0, g1, g2)
            st = np.zeros((5, 1, 1, 2, 2))
            st[:, 0, 0, 0, 0] = st[:, 0, 0, 1, 0] = c.real / 2.0
            obs = orc.observables(st, cfg)
            worst = max(worst, abs(abs(complex(obs["singlet_re"], obs["singlet_im"])) - a00))
    return worst


# ----------------------------------------------------------------- exponential

def pin_expm(orc, trials=20):
    """exp(-i delta V) against scipy.linalg.expm, plus unitarity and the eigen-reconstruction."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for t in range(trials):
        A = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
        V = (A + A.conj().T) * (0.05 if t % 2 else 1.0)
        if t == 3:                                   # degenerate spectrum
            V = np.diag([0.3, 0.3, -0.1, -0.1, 0.3]).astype(complex)
        delta = [1.0, 0.25, 0.125, 2.0][t % 4]
        U = orc.expm(V, delta)
        worst = max(worst, float(np.abs(U - sl.expm(-1j * delta * V)).max()))
        worst = max(worst, float(np.abs(U @ U.conj().T - np.eye(5)).max()))
        lam, Q = orc.heig(V)
        worst = max(worst, float(np.abs(Q @ np.diag(lam) @ Q.conj().T - V).max()))
    return worst


# ----------------------------------------------------------------- kinetic operator

def kinetic_symbol(kx, ky=None, variant=0):
    """Fourier symbol (2x2, acting on (a_m, b_m)) of the kinetic operator for a plane wave
    e^{i(kx x + ky y)}: S_q (q(j) <- q(j-1)) multiplies qubit q by e^{-ik}, S^T_q by e^{+ik};
    block I'_q = S_q C' S^T_q C; one axis is I'_1 I'_1 I'_2 I'_2 (Sec. VII.B)."""
    first, second = collide_pair(variant)

    def axis(k):
        def S(q, d):
            M = np.eye(2, dtype=complex)
            M[q, q] = np.exp(-1j * d * k)
            return M

        def block(q):
            return S(q, +1) @ second @ S(q, -1) @ first
        return block(0) @ block(0) @ block(1) @ block(1)
    K = axis(kx)
    if ky is not None:
        K = axis(ky) @ K
    return K


def pin_plane_wave_symbol(orc, variant=0):
    """The oracle's kinetic operator on every plane wave of a small 1D and 2D lattice equals
    the closed-form symbol product."""
    rng = np.random.default_rng(11)
    worst = 0.0
    L = 12
    for n in range(L):
        k = 2 * np.pi * n / L
        A = rng.normal(size=(5, 2)) + 1j * rng.normal(size=(5, 2))
        j = np.arange(L)
        field = A[:, None, None, :] * np.exp(1j * k * j)[None, None, :, None]
        st = np.stack([field.real, field.imag], axis=-1).copy()
        cfg = oracle.make_cfg(1, L, 1, 0, 0, 0, kinetic_variant=variant)
        orc.apply_kinetic(st, cfg)
        got = st[..., 0] + 1j * st[..., 1]
        want = (A @ kinetic_symbol(k, variant=variant).T)[:, None, None, :] * \
            np.exp(1j * k * j)[None, None, :, None]
        worst = max(worst, float(np.abs(got - want).max()))
    nx, ny = 6, 5
    for nxw in range(nx):
        for nyw in range(ny):
            kx, ky = 2 * np.pi * nxw / nx, 2 * np.pi * nyw / ny
            A = rng.normal(size=(5, 2)) + 1j * rng.normal(size=(5, 2))
            ph = np.exp(1j * (kx * np.arange(nx)[None, :] + ky * np.arange(ny)[:, None]))
            field = A[:, None, None, :] * ph[None, :, :, None]
            st = np.stack([field.real, field.imag], axis=-1).copy()
            cfg = oracle.make_cfg(2, nx, ny, 0, 0, 0, kinetic_variant=variant)
            orc.apply_kinetic(st, cfg)
            got = st[..., 0] + 1j * st[..., 1]
            want = (A @ kinetic_symbol(kx, ky, variant=variant).T)[:, None, None, :] * \
                ph[None, :, :, None]
            worst = max(worst, float(np.abs(got - want).max()))
    return worst


def kinetic_phase_error(orc, variant=0, L=2048):
    """Sec. VII.B: the kinetic operator is psi - i p^2 psi + O(p^4) on the boson (a = b)
    mode.  Returns max over small kappa of |(<s|K s> - 1)/kappa^2 + i| / kappa^2."""
    worst = 0.0
    for n in (1, 2, 4, 8):
        k = 2 * np.pi * n / L
        j = np.arange(L)
        w = np.exp(1j * k * j)
        st = np.zeros((5, 1, L, 2, 2))
        for q in (0, 1):
            st[2, 0, :, q, 0] = w.real / np.sqrt(2)
            st[2, 0, :, q, 1] = w.imag / np.sqrt(2)
        cfg = oracle.make_cfg(1, L, 1, 0, 0, 0, kinetic_variant=variant)
        orc.apply_kinetic(st, cfg)
        a = st[2, 0, :, 0, 0] + 1j * st[2, 0, :, 0, 1]
        b = st[2, 0, :, 1, 0] + 1j * st[2, 0, :, 1, 1]
        amp = np.mean((a + b) / np.sqrt(2) * np.conj(w))        # <s| K |s> for the plane wave
        worst = max(worst, abs((amp - 1.0) / k ** 2 + 1j) / k ** 2)
    return worst


# ----------------------------------------------------------------- dense brute force

def _vec(st):
    return (st[..., 0] + 1j * st[..., 1]).reshape(-1)


def _unvec(v, shape):
    z = v.reshape(shape[:-1])
    return np.stack([z.real, z.imag], axis=-1)


def dense_collide(N, C):
    D = np.zeros((10 * N, 10 * N), dtype=complex)
    for m in range(5):
        for s in range(N):
            i0 = (m * N + s) * 2
            D[i0:i0 + 2, i0:i0 + 2] = C
    return D


def dense_stream(nx, ny, axis, q, d):
    """Permutation: qubit q of every level moves one site toward +axis (d=+1) or -axis."""
    N = nx * ny
    P = np.zeros((10 * N, 10 * N))
    for m in range(5):
        for y in range(ny):
            for x in range(nx):
                s = y * nx + x
                for qq in (0, 1):
                    if qq == q:
                        sx, sy = ((x - d) % nx, y) if axis == 0 else (x, (y - d) % ny)
                    else:
                        sx, sy = x, y
                    P[(m * N + s) * 2 + qq, (m * N + sy * nx + sx) * 2 + qq] = 1.0
    return P


def dense_potential(orc, v, N, g, delta):
    """Block-diagonal U = exp(-i delta V(psi_site)) acting on the level index of each qubit;
    V from the (Table I-pinned) oracle matrix, the exponential from scipy."""
    z = v.reshape(5, N, 2)
    D = np.zeros((10 * N, 10 * N), dtype=complex)
    for s in range(N):
        psi = z[:, s, 0] + z[:, s, 1]
        Us = sl.expm(-1j * delta * orc.potential_matrix(psi, *g))
        for q in (0, 1):
            idx = [(m * N + s) * 2 + q for m in range(5)]
            D[np.ix_(idx, idx)] = Us
    return D


def pin_dense_step(orc, ndim, interleave=0, variant=0, nsteps=2, seed=3):
    """One oracle step against the product of dense operator matrices on a tiny lattice
    (L = 4 in 1D, 3 x 3 in 2D) with random amplitudes and couplings."""
    rng = np.random.default_rng(seed)
    nx, ny = (4, 1) if ndim == 1 else (3, 3)
    N = nx * ny
    g = tuple(rng.uniform(-1, 1, size=3))
    st = 0.3 * rng.normal(size=(5, ny, nx, 2, 2))
    cfg = oracle.make_cfg(ndim, nx, ny, *g, interleave=interleave, kinetic_variant=variant)
    first, second = collide_pair(variant)
    C1, C2 = dense_collide(N, first), dense_collide(N, second)
    v = _vec(st)
    for _ in range(nsteps):
        blocks = []
        for axis in range(ndim):
            for q in (1, 1, 0, 0):
                blocks.append(dense_stream(nx, ny, axis, q, +1) @ C2 @
                              dense_stream(nx, ny, axis, q, -1) @ C1)
        if not interleave:
            v = dense_potential(orc, v, N, g, 1.0) @ v
            for B in blocks:
                v = B @ v
        else:
            for B in blocks:
                v = dense_potential(orc, v, N, g, 1.0 / (4 * ndim)) @ v
                v = B @ v
    orc.step(st, cfg, nsteps)
    return float(np.abs(_vec(st) - v).max())


# ----------------------------------------------------------------- exact Thomas-Fermi phase

def pin_tf_phase(orc, interleave=0, nsteps=3):
    """A uniform Table I state with a = b = c/2 is an exact eigenvector of one QLGA step:
    the kinetic operator is the identity on it (zero wavenumber, a = b) and V(c) c = E c, so
    n steps multiply it by exp(-i E n) exactly."""
    worst = 0.0
    for E, g0, g1, g2 in COUPLING_SETS[:3]:
        Elat = 0.02 * E                   # lattice energy: small field, as after eps-scaling
        for row, c in golden.table1(Elat, g0, g1, g2, c1=0.03, c2=0.02).items():
            c = np.asarray(c)
            for ndim, (nx, ny) in ((1, (8, 1)), (2, (4, 3))):
                st = np.zeros((5, ny, nx, 2, 2))
                st[..., 0, 0] = st[..., 1, 0] = (c / 2.0)[:, None, None]
                want = np.exp(-1j * Elat * nsteps) * _vec(st)
                cfg = oracle.make_cfg(ndim, nx, ny, g0, g1, g2, interleave=interleave)
                orc.step(st, cfg, nsteps)
                worst = max(worst, float(np.abs(_vec(st) - want).max()) / max(np.abs(c).max(), 1e-300))
    return worst


def pin_norm(orc, ndim=2, nsteps=4):
    """Unitarity: the qubit norm after nsteps of a random state, relative drift."""
    rng = np.random.default_rng(5)
    nx, ny = (7, 1) if ndim == 1 else (6, 5)
    st = 0.2 * rng.normal(size=(5, ny, nx, 2, 2))
    cfg = oracle.make_cfg(ndim, nx, ny, 1.0, 0.8, -0.6)
    n0 = float((st ** 2).sum())
    orc.step(st, cfg, nsteps)
    return abs(float((st ** 2).sum()) - n0) / n0


# ----------------------------------------------------------------- observables

def _uniform_state(c, nx, ny):
    """a = b = c / 2 on every site of an nx x ny lattice (c complex, 5 levels)."""
    st = np.zeros((5, ny, nx, 2, 2))
    for q in (0, 1):
        st[..., q, 0] = (np.real(c) / 2)[:, None, None]
        st[..., q, 1] = (np.imag(c) / 2)[:, None, None]
    return st


def pin_observables(orc):
    """Observables against closed forms (Sec. III.B Eq. cmap, Sec. IV.B).  Uniform Thomas-Fermi
    rows (Table I) turned by a global phase phi: the energy density is E rho / 2 (c^dagger V(c) c
    = E rho for an eigenvector of V), the qubit populations |c_m|^2 / 2, the magnetisation
    sum_m m |c_m|^2 / 2, the qubit norm rho / 2 per site, and the overlap with the same state
    turned by alpha is N rho e^{i alpha}; row 5 (m = 0 only) has the singlet sum
    N c_0^2 e^{2 i phi} / sqrt(5) and singlet fraction 1, row 1 (m = +2 only) neither.  Plane
    waves A e^{i k x} along x and along y carry the forward-difference kinetic energy
    2 |A|^2 (1 - cos k) per site."""
    worst = 0.0
    E, g0, g1, g2 = 0.02, 1.0, 0.1, 1.0
    nx, ny = 4, 3
    N = nx * ny
    phi, alpha = 0.7, -1.1
    ms = np.array([2.0, 1.0, 0.0, -1.0, -2.0])
    for row, c in golden.table1(E, g0, g1, g2, c1=0.03, c2=0.02).items():
        c = np.asarray(c, dtype=float) * np.exp(1j * phi)
        st = _uniform_state(c, nx, ny)
        ref = _uniform_state(c * np.exp(1j * alpha), nx, ny)
        o = orc.observables(st, oracle.make_cfg(2, nx, ny, g0, g1, g2), ref=ref)
        p = np.abs(c) ** 2
        rho = float(p.sum())
        dev = [o["energy"] - N * E * rho / 2, o["magnetisation"] - N * float(ms @ p) / 2,
               o["norm_boson"] - N * rho, o["norm_qubit"] - N * rho / 2,
               complex(o["overlap_re"], o["overlap_im"]) - N * rho * np.exp(1j * alpha)]
        dev += list(o["pop"] - N * p / 2)
        if row == 5:
            dev += [complex(o["singlet_re"], o["singlet_im"]) - N * c[2] ** 2 / np.sqrt(5),
                    o["singlet_fraction"] - 1.0]
        if row == 1:
            dev += [complex(o["singlet_re"], o["singlet_im"]), o["singlet_fraction"]]
        worst = max(worst, max(abs(d) for d in dev))
    # plane waves in level +1, along x and along y
    nx, ny = 16, 8
    A = 0.3 + 0.1j
    for axis, n_axis in ((0, nx), (1, ny)):
        k = 2 * np.pi * 3 / n_axis
        j = np.arange(n_axis)
        w = A * np.exp(1j * k * j) / 2
        grid = w[None, :] * np.ones((ny, 1)) if axis == 0 else w[:, None] * np.ones((1, nx))
        st = np.zeros((5, ny, nx, 2, 2))
        for q in (0, 1):
            st[1, ..., q, 0] = grid.real
            st[1, ..., q, 1] = grid.imag
        o = orc.observables(st, oracle.make_cfg(2, nx, ny, 0, 0, 0))
        worst = max(worst, abs(o["energy"] - nx * ny * 2 * abs(A) ** 2 * (1 - np.cos(k))))
    return worst


# ----------------------------------------------------------------- per-site fields

def pin_fields(orc):
    """Per-site fields: Table II values on uniform Thomas-Fermi lattices (Sec. III.B), unit colour
    vectors (Eq. colormap), zero vorticity for a plane wave, the discrete curl summing to exactly
    zero over the torus, and +-2 pi around a vortex / antivortex (Sec. VI.B)."""
    from paper_1907_12834_gb300 import inputs
    worst = 0.0
    E, g0, g1, g2 = 1.0, 1.0, 0.1, 1.0
    rows1 = golden.table1(E, g0, g1, g2)
    for row, ((fpar, fperp, a00), flags) in golden.table2(E, g0, g1, g2).items():
        if row not in rows1:
            continue
        c = np.asarray(rows1[row])
        st = np.zeros((5, 4, 4, 2, 2))
        st[..., 0, 0] = st[..., 1, 0] = (c / 2.0)[:, None, None]
        f = orc.fields(st, oracle.make_cfg(2, 4, 4, g0, g1, g2))
        worst = max(worst, float(np.abs(np.abs(f[0]) - fpar).max()), float(np.abs(f[2] - a00).max()))
        if "perp-misprint" not in flags:
            worst = max(worst, float(np.abs(f[1] - fperp).max()))
        nrm = np.sqrt(f[3] ** 2 + f[4] ** 2 + f[5] ** 2)
        worst = max(worst, float(np.abs(nrm[nrm > 0] - 1.0).max(initial=0.0)))
    # plane wave in level +1: no vorticity
    nx, ny = 32, 16
    k = 2 * np.pi * 3 / nx
    st = np.zeros((5, ny, nx, 2, 2))
    w = 0.05 * np.exp(1j * k * np.arange(nx))[None, :] * np.ones((ny, 1))
    st[1, ..., 0, 0] = st[1, ..., 1, 0] = w.real
    st[1, ..., 0, 1] = st[1, ..., 1, 1] = w.imag
    f = orc.fields(st, oracle.make_cfg(2, nx, ny, g0, g1, g2))
    worst = max(worst, float(np.abs(f[6:]).max()))
    # vortex dipole in level +2: +2 pi around the vortex, -2 pi around the antivortex, 0 in total
    n = 96
    psi = np.zeros((5, n, n), complex)
    psi[0] = inputs.vortex_dipole(n, n, 0.1, 2, (g0, g1, g2), separation=40.0)
    st = inputs.boson_to_state(psi, 0.1)
    f = orc.fields(st, oracle.make_cfg(2, n, n, g0, g1, g2))
    om = f[6]
    worst = max(worst, abs(float(om.sum())))
    cx, cy = int(n / 2 + 0.5), int(n / 2 + 0.5)
    # the sum of the central-difference curl over a box telescopes to a closed loop of wrapped
    # phase differences: exactly 2 pi times the winding inside
    box = lambda xc, h: om[cy - h:cy + h + 1, xc - h:xc + h + 1].sum()
    for h in (4, 12):
        worst = max(worst, abs(box(cx - 20, h) - 2 * np.pi), abs(box(cx + 20, h) + 2 * np.pi))
    return worst


# ----------------------------------------------------------------- adjoint (reverse mode)

def _rand_state(rng, ndim, nx, ny, amp=0.35):
    shape = (5, ny, nx, 2, 2)
    return np.ascontiguousarray(amp * rng.standard_normal(shape))


def pin_frechet(orc, trials=12, seed=11):
    """max relative deviation of L(-i delta V, E) from the upper-right block of
    exp([[A, E], [0, A]]) with A = -i delta V (the block-triangular identity for the Frechet
    derivative of the matrix exponential), scipy's expm.  V: random Hermitian matrices, the
    potential of random sites, and a degenerate V (repeated eigenvalues)."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    cases = []
    for t in range(trials):
        X = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
        cases.append((0.5 * (X + X.conj().T), 0.3 + 0.2 * t))
        psi = 0.6 * (rng.standard_normal(5) + 1j * rng.standard_normal(5))
        cases.append((orc.potential_matrix(psi, 1.0, -0.5 + 0.1 * t, 0.7 - 0.15 * t), 1.0))
    cases.append((np.diag([1.0, 1.0, -0.5, 2.0, 2.0]).astype(complex), 1.0))
    for V, delta in cases:
        E = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
        A = -1j * delta * V
        big = np.zeros((10, 10), dtype=complex)
        big[:5, :5] = A
        big[5:, 5:] = A
        big[:5, 5:] = E
        ref = sl.expm(big)[:5, 5:]
        got = orc.frechet_exp(V, delta, E)
        worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    return worst


def _dot(u, v):
    return float(np.sum(u * v))


def pin_kinetic_adjoint(orc):
    """max relative violation of <K v, w> = <v, K^dagger w> (real inner product of the state
    buffers, i.e. Re sum conj(x) y) and of K^dagger K v = v (K is unitary), 1D and 2D, K1/K2."""
    rng = np.random.default_rng(5)
    worst = 0.0
    for ndim, nx, ny in ((1, 12, 1), (2, 7, 6)):
        for variant in (0, 1):
            cfg = oracle.make_cfg(ndim, nx, ny, 1.0, 0.2, 0.3, kinetic_variant=variant)
            v = _rand_state(rng, ndim, nx, ny)
            w = _rand_state(rng, ndim, nx, ny)
            Kv = orc.apply_kinetic(v.copy(), cfg)
            Ktw = orc.vjp_kinetic(w.copy(), cfg)
            lhs, rhs = _dot(Kv, w), _dot(v, Ktw)
            worst = max(worst, abs(lhs - rhs) / (np.linalg.norm(v) * np.linalg.norm(w)))
            back = orc.vjp_kinetic(Kv.copy(), cfg)
            worst = max(worst, float(np.abs(back - v).max()))
    return worst


def _fd_directional(fwd, x, v, h):
    """Central difference of the map fwd at x in direction v (fourth order: two step sizes)."""
    d1 = (fwd(x + h * v) - fwd(x - h * v)) / (2 * h)
    d2 = (fwd(x + 2 * h * v) - fwd(x - 2 * h * v)) / (4 * h)
    return (4 * d1 - d2) / 3


ADJ_CASES = [  # (ndim, nx, ny, (g0, g1, g2), variant)
    (1, 10, 1, (1.0, -0.5, 0.2), 0),
    (1, 9, 1, (1.0, 0.8, -0.6), 1),
    (2, 6, 5, (1.0, 0.1, 1.0), 0),
    (2, 5, 6, (0.7, -0.4, 0.9), 1),
]


def pin_vjp_fd(orc, what="step", nsteps=3, seed=21):
    """max relative deviation between <vjp(w), v> and <w, J v>, J v the central finite
    difference of the forward map in a random direction v, for w a random cotangent.
    what: "potential" (U alone, delta = 1 and 1/4), "step" (one plain step) or "run" (nsteps
    plain steps through vjp_run).  The forward operators are pinned independently."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for ndim, nx, ny, g, variant in ADJ_CASES:
        cfg = oracle.make_cfg(ndim, nx, ny, *g, kinetic_variant=variant)
        x = _rand_state(rng, ndim, nx, ny)
        v = _rand_state(rng, ndim, nx, ny, amp=1.0)
        w = _rand_state(rng, ndim, nx, ny, amp=1.0)
        deltas = (1.0, 0.25) if what == "potential" else (1.0,)
        for delta in deltas:
            if what == "potential":
                fwd = lambda s: orc.apply_potential(np.ascontiguousarray(s), cfg, delta)
                cot = w.copy()
                orc.vjp_potential(x, cot, cfg, delta)
            elif what == "step":
                fwd = lambda s: orc.step(np.ascontiguousarray(s), cfg, 1)
                cot = w.copy()
                orc.vjp_step(x, cot, cfg)
            else:
                fwd = lambda s: orc.step(np.ascontiguousarray(s), cfg, nsteps)
                cot = w.copy()
                orc.vjp_run(x, nsteps, cot, cfg)
            jv = _fd_directional(fwd, x, v, 1e-5)
            lhs, rhs = _dot(w, jv), _dot(cot, v)
            worst = max(worst, abs(lhs - rhs) / max(abs(lhs), 1e-3 * np.linalg.norm(w) * np.linalg.norm(v)))
    return worst


def pin_coupling_fd(orc, nsteps=3, seed=23):
    """max relative deviation of dL/dg from vjp_run against central finite differences in each
    coupling, L = <w, x_n> for a random cotangent w."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for ndim, nx, ny, g, variant in ADJ_CASES:
        x = _rand_state(rng, ndim, nx, ny)
        w = _rand_state(rng, ndim, nx, ny, amp=1.0)
        cfg = oracle.make_cfg(ndim, nx, ny, *g, kinetic_variant=variant)
        cot = w.copy()
        dg = orc.vjp_run(x, nsteps, cot, cfg)

        def loss(gv):
            c = oracle.make_cfg(ndim, nx, ny, *gv, kinetic_variant=variant)
            return _dot(w, orc.step(x.copy(), c, nsteps))

        h = 1e-5
        for i in range(3):
            e = np.zeros(3)
            e[i] = 1.0
            gp = np.array(g)
            d1 = (loss(gp + h * e) - loss(gp - h * e)) / (2 * h)
            d2 = (loss(gp + 2 * h * e) - loss(gp - 2 * h * e)) / (4 * h)
            fd = (4 * d1 - d2) / 3
            worst = max(worst, abs(fd - dg[i]) / max(abs(fd), 1e-3))
    return worst


def pin_tf_coupling_gradient(orc):
    """Closed form: a uniform single-level state psi = (c, 0, 0, 0, 0) with a = b = psi/2 is an
    eigenvector of V with eigenvalue (g0 + 4 g1) rho and is left alone by the kinetic operator
    (zero momentum), so one step is x' = exp(-i (g0 + 4 g1) rho) x.  For L = <w, x'>:
    dL/dg0 = <w, -i rho x'>, dL/dg1 = 4 dL/dg0, dL/dg2 = 0.  Returns the max relative deviation."""
    rng = np.random.default_rng(29)
    worst = 0.0
    for ndim, nx, ny in ((1, 8, 1), (2, 6, 6)):
        for g in ((1.0, -0.5, 0.2), (0.6, 0.3, -0.8)):
            cfg = oracle.make_cfg(ndim, nx, ny, *g)
            c = 0.45 * np.exp(0.7j)
            x = np.zeros((5, ny, nx, 2, 2))
            x[0, :, :, :, 0] = c.real / 2
            x[0, :, :, :, 1] = c.imag / 2
            rho = abs(c) ** 2
            theta = (g[0] + 4 * g[1]) * rho
            xc = x[..., 0] + 1j * x[..., 1]
            xp = np.exp(-1j * theta) * xc
            w = rng.standard_normal(x.shape)
            wc = w[..., 0] + 1j * w[..., 1]
            dg0 = float(np.sum((np.conj(wc) * (-1j * rho) * xp).real))
            cot = w.copy()
            dg = orc.vjp_step(x, cot, cfg)
            ref = np.array([dg0, 4 * dg0, 0.0])
            worst = max(worst, float(np.abs(dg - ref).max() / abs(dg0)))
    return worst
