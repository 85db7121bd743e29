"""Seeded synthetic inputs: the paper's analytic spin-2 states, mapped to the QLGA state.

This module only builds initial states.  It holds none of the time-step arithmetic, and
both the CUDA library and the CPU oracle consume what it returns (NumPy arrays).

* Thomas-Fermi / soliton coefficients: Table I (Sec. III.A).  Bright soliton
  psi_m = c_m k sech(k x) with the Table I coefficients at E = -2, eigenvalue -k^2
  (Sec. III.C, Eq. system_of_equations_bright); dark soliton c_m k tanh(k x) with E = 2
  (Eq. system_of_equations_kinks); periodic dark pair as the product of two kinks (Sec. IV.A).
* Kicks: multiply by exp(i 2 pi n x / L), n an integer (Sec. IV.B; Sec. VI.A.2 in 2D).
* Pade vortex: sqrt((a2 r^4 + a1 r^2) / (a2 r^4 + b1 r^2 + 1)) e^{i theta}
  (Eq. pade_form) with the coefficients of Table III.
* Lattice scaling: x = eps j, t = eps^2 n, phi = eps psi (Sec. VII.A, Eq. eomscaling), split
  into the qubit pair as a = b = phi / 2.

State arrays have shape (5, ny, nx, 2, 2): level m = +2..-2, y, x, qubit (a, b), (re, im).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

M_VALUES = (2, 1, 0, -1, -2)


# --------------------------------------------------------------------------- Table I

def table1_coefficients(row: int, E: float, g0: float, g1: float, g2: float,
                        c1: float | None = None, c2: float | None = None) -> np.ndarray:
    """Coefficients (c_2, c_1, c_0, c_-1, c_-2) of Table I row `row` (1..16).

    Rows 11, 12 and 16 are one-parameter families; c1 / c2 are their free coefficients.
    Raises ValueError when the couplings make a coefficient non-real (the table only holds
    where every c_m is real, per its caption).
    """
    q = _real_sqrt
    if row == 1:
        c = [q(E / (g0 + 4 * g1)), 0, 0, 0, 0]
    elif row == 2:
        c = [0, 0, 0, 0, q(E / (g0 + 4 * g1))]
    elif row == 3:
        c = [0, q(E / (g0 + g1)), 0, 0, 0]
    elif row == 4:
        c = [0, 0, 0, q(E / (g0 + g1)), 0]
    elif row == 5:
        c = [0, 0, q(5 * E / (5 * g0 + g2)), 0, 0]
    elif row == 6:
        v = q(5 * E / (10 * g0 + 2 * g2))
        c = [v, 0, 0, 0, v]
    elif row == 7:
        v = q(5 * E / (10 * g0 + 2 * g2))
        c = [0, v, 0, v, 0]
    elif row == 8:
        c = [q(E / (3 * g0)), 0, 0, q(2 * E / (3 * g0)), 0]
    elif row == 9:
        c = [0, q(2 * E / (3 * g0)), 0, 0, q(E / (3 * g0))]
    elif row == 10:
        c = [q(E / (4 * g0)), 0, q(E / (2 * g0)), 0, -q(E / (4 * g0))]
    elif row == 11:
        c2 = _need(c2, "c2")
        c = [c2, 0, q((5 * E - 10 * c2 ** 2 * g0 - 2 * c2 ** 2 * g2) / (5 * g0 + g2)), 0, c2]
    elif row == 12:
        c1 = _need(c1, "c1")
        c = [0, c1, q((5 * E - 10 * c1 ** 2 * g0 - 2 * c1 ** 2 * g2) / (5 * g0 + g2)), -c1, 0]
    elif row == 13:
        v = q(E / (4 * g0 + 4 * g1))
        c = [v, v, 0, -v, -v]
    elif row == 14:
        c = [q(3 * E / (16 * g0)), q(E / (4 * g0)), -q(E / (8 * g0)), q(E / (4 * g0)),
             q(3 * E / (16 * g0))]
    elif row == 15:
        v = q(E / (g0 + 4 * g1))
        c = [v / 4, v / 2, 0.5 * q(3 * E / (2 * g0 + 8 * g1)), v / 2, v / 4]
    elif row == 16:
        c1 = _need(c1, "c1")
        c2 = _need(c2, "c2")
        c = [c2, c1, q((5 * E - (c2 ** 2 + c1 ** 2) * (10 * g0 + 2 * g2)) / (5 * g0 + g2)), -c1, c2]
    else:
        raise ValueError("Table I has rows 1..16")
    return np.asarray(c, dtype=np.float64)


def _real_sqrt(v: float) -> float:
    if not np.isfinite(v) or v < 0:
        raise ValueError("coefficient is not real for these couplings")
    return math.sqrt(v)


def _need(v, name):
    if v is None:
        raise ValueError("this Table I row needs its free coefficient %s" % name)
    return float(v)


# --------------------------------------------------------------------------- Table III

def pade_coefficients(mf: int, E: float, g0: float, g1: float, g2: float):
    """(a1, b1, a2) of the single-channel Pade vortex in level mf (Table III).

    Both roots of the a1 formula are tried; the one with a1, b1, a2 > 0 and b1 > a1 (the
    condition Sec. VI.A states for a tanh-like profile) is returned.
    """
    roots = []
    for sign in (+1.0, -1.0):
        if abs(mf) == 2:
            G = g0 + 4 * g1
            gam = E ** 2 * math.sqrt(361 * E ** 2 - 8 * G * (4 * G + 13 * E))
            a1 = (19 * E ** 3 - 12 * G * E ** 2 + sign * gam) / (64 * G * (2 * E - G))
            b1 = (16 * a1 * (G - 3 * E) + 5 * E ** 2) / (48 * (E - 4 * a1))
        elif abs(mf) == 1:
            G = g0 + g1
            gam = E ** 2 * math.sqrt(361 * E ** 2 - 8 * G * (4 * G + 13 * E))
            a1 = -11 * E ** 4 / (76 * E ** 3 - 48 * G * E ** 2 + sign * 4 * gam)
            b1 = (16 * a1 * (G - 3 * E) + 5 * E ** 2) / (48 * (E - 4 * a1))
        elif mf == 0:
            G = 5 * g0 + g2
            gam = E ** 2 * math.sqrt(9025 * E ** 2 - 8 * G * (20 * g0 + 4 * g2 + 65 * E))
            a1 = 5 * (95 * E ** 3 - 12 * G * E ** 2 + sign * gam) / (64 * G * (10 * E - G))
            b1 = (16 * a1 * (G - 15 * E) + 25 * E ** 2) / (240 * (E - 4 * a1))
        else:
            raise ValueError("mf must be in -2..2")
        a2 = a1 * (b1 - E / 4)
        roots.append((a1, b1, a2))
    for a1, b1, a2 in roots:
        if a1 > 0 and b1 > 0 and a2 > 0 and b1 > a1:
            return a1, b1, a2
    raise ValueError("no Table III root with b1 > a1 > 0 for these couplings")


def pade_profile(r: np.ndarray, a1: float, b1: float, a2: float) -> np.ndarray:
    """|psi| of Eq. pade_form at physical radius r."""
    r2 = r * r
    return np.sqrt((a2 * r2 * r2 + a1 * r2) / (a2 * r2 * r2 + b1 * r2 + 1.0))


# --------------------------------------------------------------------------- mapping

def boson_to_state(psi: np.ndarray, eps: float, dtype=np.float64) -> np.ndarray:
    """Physical boson field psi[5, ny, nx] (complex) -> QLGA state, a = b = eps psi / 2."""
    psi = np.asarray(psi)
    if psi.ndim == 2:
        psi = psi[:, None, :]
    phi = (0.5 * eps) * psi
    st = np.empty(psi.shape + (2, 2), dtype=dtype)
    st[..., 0, 0] = phi.real
    st[..., 0, 1] = phi.imag
    st[..., 1, 0] = phi.real
    st[..., 1, 1] = phi.imag
    return st


def state_to_boson(state: np.ndarray) -> np.ndarray:
    """QLGA state -> lattice boson field psi_m = a_m + b_m, complex [5, ny, nx]."""
    s = np.asarray(state, dtype=np.float64)
    return (s[..., 0, 0] + s[..., 1, 0]) + 1j * (s[..., 0, 1] + s[..., 1, 1])


def random_state(rng: np.random.Generator, nx: int, ny: int = 1, scale: float = 0.05,
                 dtype=np.float64) -> np.ndarray:
    """Independent Gaussian amplitudes of size `scale` on every qubit (parity-test input)."""
    return (scale * rng.standard_normal((5, ny, nx, 2, 2))).astype(dtype)


# --------------------------------------------------------------------------- 1D states

def bright_soliton(x: np.ndarray, row: int, g: tuple, k: float = 1.0, x0: float = 0.0,
                   p: float = 0.0, phase: float = 0.0, c1=None, c2=None) -> np.ndarray:
    """psi_m(x) = c_m k sech(k (x - x0)) e^{i p x + i phase}, c from Table I at E = -2."""
    c = table1_coefficients(row, -2.0, *g, c1=c1, c2=c2)
    u = np.abs(k * (x - x0))
    prof = k * 2.0 * np.exp(-u) / (1.0 + np.exp(-2.0 * u))      # k sech(u), overflow-free
    return c[:, None] * prof[None, :] * np.exp(1j * (p * x + phase))[None, :]


def dark_soliton_pair(x: np.ndarray, L: float, row: int, g: tuple, k: float = 1.0,
                      c1=None, c2=None) -> np.ndarray:
    """Periodic dark-soliton pair: c_m k tanh(k (x - L/4)) tanh(k (3L/4 - x)), c at E = 2."""
    c = table1_coefficients(row, 2.0, *g, c1=c1, c2=c2)
    prof = k * np.tanh(k * (x - 0.25 * L)) * np.tanh(k * (0.75 * L - x))
    return c[:, None] * prof[None, :]


# --------------------------------------------------------------------------- 2D states

def vortex_dipole_phase(nx: int, ny: int, x1: float, x2: float, yc: float) -> np.ndarray:
    """Phase of a vortex (+1) at (x1, yc) and an antivortex (-1) at (x2, yc), lattice units.

    arg[ sin(pi (z - z1) / nx) / sin(pi (z - z2) / nx) ] is periodic in x; the linear term
    removes the 2 pi (x1 - x2) / nx step it leaves across the y boundary.
    """
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    z = x + 1j * (y - yc)
    num = np.sin(np.pi * (z - x1) / nx)
    den = np.sin(np.pi * (z - x2) / nx)
    th = np.angle(num / den)
    d = x1 - x2
    corr = -2.0 * np.pi * d / nx * (y / ny) + np.pi * d / nx
    return th + corr


def vortex_dipole(nx: int, ny: int, eps: float, mf: int, g: tuple, E: float = 1.0,
                  separation: float = 64.0, winding: int = +1, kick=(0, 0)) -> np.ndarray:
    """One level's field: Pade vortex and antivortex `separation` sites apart along x at the
    lattice centre, unit background, optional integer kick (n_x, n_y)."""
    a1, b1, a2 = pade_coefficients(mf, E, *g)
    # cores sit half a site off the lattice points, so that no site falls on a phase singularity
    cx, cy = nx / 2.0 + 0.5, ny / 2.0 + 0.5
    x1, x2 = cx - separation / 2.0, cx + separation / 2.0
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    # nearest periodic image distance, in physical units (x = eps j)
    def dist(xc):
        dx = (x - xc + nx / 2.0) % nx - nx / 2.0
        dy = (y - cy + ny / 2.0) % ny - ny / 2.0
        return eps * np.sqrt(dx * dx + dy * dy)
    amp = pade_profile(dist(x1), a1, b1, a2) * pade_profile(dist(x2), a1, b1, a2)
    th = winding * vortex_dipole_phase(nx, ny, x1, x2, cy)
    th = th + 2.0 * np.pi * (kick[0] * x / nx + kick[1] * y / ny)
    return amp * np.exp(1j * th)


# --------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    ndim: int
    nx: int
    ny: int
    g: tuple
    eps: float
    steps: int
    precision: int
    state: np.ndarray = field(repr=False)
    meta: dict = field(default_factory=dict)


CONFIG0_G = (1.0, -0.5, 0.2)


def config0(row: int = 1, L: int = 1024, eps: float = 0.1, steps: int = 2000) -> Workload:
    """1D stationary bright soliton, Table I row `row` (default 1), L = 1024, FP64."""
    j = np.arange(L, dtype=np.float64)
    psi = bright_soliton(eps * (j - L / 2), row, CONFIG0_G, k=1.0)
    return Workload("1d-bright-soliton-L%d" % L, 1, L, 1, CONFIG0_G, eps, steps, 64,
                    boson_to_state(psi, eps), {"row": row})


def config1(seed: int = 1908, L: int = 16384, eps: float = 0.1, steps: int = 20000,
            couplings: tuple = CONFIG0_G, precision: int = 64) -> Workload:
    """1D two-soliton scattering, L = 16384: bright solitons of distinct Table I rows drawn
    from {1, 2, 15} (real at the profile couplings (1, -0.5, 0.2)) at L/4 and 3L/4 with
    kicks +-2 pi n / L, n = round(kappa L / 2 pi), kappa ~ U[0.05, 0.3] rad/site, and a
    relative phase ~ U[0, 2 pi).  Evolved under `couplings`."""
    rng = np.random.default_rng(seed)
    rows = rng.choice([1, 2, 15], size=2, replace=False)
    kappa = rng.uniform(0.05, 0.3)
    n = int(round(kappa * L / (2 * np.pi)))
    rel = rng.uniform(0.0, 2 * np.pi)
    j = np.arange(L, dtype=np.float64)
    p_lat = 2 * np.pi * n / L                       # rad / site
    # kicks written on the absolute lattice coordinate so that they are exactly periodic
    s1 = bright_soliton(eps * (j - L / 4), int(rows[0]), CONFIG0_G)
    s2 = bright_soliton(eps * (j - 3 * L / 4), int(rows[1]), CONFIG0_G)
    psi = s1 * np.exp(1j * p_lat * j)[None, :] + s2 * np.exp(-1j * p_lat * j + 1j * rel)[None, :]
    return Workload("1d-soliton-scattering-L%d" % L, 1, L, 1, tuple(couplings), eps, steps,
                    precision, boson_to_state(psi, eps),
                    {"rows": [int(r) for r in rows], "n_kick": n, "rel_phase": rel})


CONFIG2_G = (1.0, 0.1, 1.0)


def config2(seed: int = 1909, n: int = 4096, eps: float = 0.1, steps: int = 5000,
            variant: str = "a", separation: float = 64.0, dtype=np.float32) -> Workload:
    """2D vortex scattering on an n x n lattice (default 4096^2), FP32 state.

    Variant a: m = +2 holds a vortex / antivortex dipole, m = -2 the counter-rotating one;
    b: the same in m = +1 / -1; c: one dipole in m = 0.  Unit background, Pade cores of
    Table III at the couplings of Sec. VI.C (g0, g1, g2) = (1, 0.1, 1), E = 1, seeded
    integer kicks (n_x, n_y) in -3..3 per occupied level.
    """
    rng = np.random.default_rng(seed)
    levels = {"a": (2, -2), "b": (1, -1), "c": (0,)}[variant]
    psi = np.zeros((5, n, n), dtype=np.complex128)
    for k, mf in enumerate(levels):
        kick = tuple(int(v) for v in rng.integers(-3, 4, size=2))
        wind = +1 if k == 0 else -1
        psi[2 - mf] = vortex_dipole(n, n, eps, mf, CONFIG2_G, separation=separation,
                                    winding=wind, kick=kick)
    st = boson_to_state(psi, eps, dtype=dtype)
    del psi
    return Workload("2d-vortex-scattering-%dx%d" % (n, n), 2, n, n, CONFIG2_G, eps, steps,
                    32 if dtype == np.float32 else 64, st, {"variant": variant})


def config4(seed: int = 1911, n: int = 512, eps: float = 0.1, steps: int = 2000,
            variant: str = "a", separation: float = 64.0, dtype=np.float32) -> Workload:
    """2D vortex scattering on an n x n lattice (default 512^2), the adjoint workload: the
    recipe of config2 at its own seed, with the vortex cores 64 sites apart as in config2 (at
    separation n/64 = 8 sites the cores, about 10 sites across at eps = 0.1, would overlap)."""
    w = config2(seed=seed, n=n, eps=eps, steps=steps, variant=variant, separation=separation, dtype=dtype)
    w.meta["cores"] = dipole_cores(n, n, separation, variant)
    return w


def dipole_cores(nx: int, ny: int, separation: float, variant: str = "a"):
    """(level index, x, y) of every vortex core of a config2 / config4 state."""
    levels = {"a": (2, -2), "b": (1, -1), "c": (0,)}[variant]
    cx, cy = nx / 2.0 + 0.5, ny / 2.0 + 0.5
    out = []
    for mf in levels:
        for xc in (cx - separation / 2.0, cx + separation / 2.0):
            out.append((2 - mf, xc, cy))
    return out


def kicked_state(psi, eps, cores, velocity, phase_levels=(), phases=None, sigma=16.0, core_phases=None):
    """Differentiable initial state (torch): the boson field psi (complex numpy [5, ny, nx])
    with a windowed local kick and phase at each vortex core and a phase on some levels.

    Core j at (level l_j, x_j, y_j) gets psi_l <- psi_l exp(i (v_j . d + phi_j) w_j), d the
    nearest-image displacement from the core and w_j = exp(-|d|^2 / (2 sigma^2)): a local phase
    gradient v_j (rad / site) that moves the core with a continuous velocity, unlike the quantised
    global kicks 2 pi n / L, and a local phase phi_j (the relative phase of the cores).  Level
    phase_levels[k] is multiplied by exp(i phases[k]) (a level's global phase: for losses that are
    invariant under the global phase and under rotations about z these are symmetry directions).
    velocity: torch tensor [ncores, 2]; core_phases: torch tensor [ncores] or None; phases: torch
    tensor [len(phase_levels)].  Returns the QLGA state a = b = eps psi / 2 as a torch tensor
    (5, ny, nx, 2, 2) of velocity's dtype and device."""
    import torch
    dev, dt = velocity.device, velocity.dtype
    ny, nx = psi.shape[1], psi.shape[2]
    re = torch.tensor(np.ascontiguousarray(psi.real), dtype=dt, device=dev)
    im = torch.tensor(np.ascontiguousarray(psi.imag), dtype=dt, device=dev)
    x = torch.arange(nx, dtype=dt, device=dev)[None, :]
    y = torch.arange(ny, dtype=dt, device=dev)[:, None]
    theta = torch.zeros((5, ny, nx), dtype=dt, device=dev)
    for j, (lev, xc, yc) in enumerate(cores):
        dx = torch.remainder(x - xc + nx / 2.0, nx) - nx / 2.0
        dy = torch.remainder(y - yc + ny / 2.0, ny) - ny / 2.0
        w = torch.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))
        th = (velocity[j, 0] * dx + velocity[j, 1] * dy) * w
        if core_phases is not None:
            th = th + core_phases[j] * w
        theta = theta + torch.nn.functional.one_hot(torch.tensor(lev), 5).to(dt).to(dev)[:, None, None] * th[None]
    for k, lev in enumerate(phase_levels):
        theta = theta + torch.nn.functional.one_hot(torch.tensor(lev), 5).to(dt).to(dev)[:, None, None] * phases[k]
    c, s = torch.cos(theta), torch.sin(theta)
    pr = re * c - im * s
    pi = re * s + im * c
    half = 0.5 * eps
    a = torch.stack([half * pr, half * pi], dim=-1)
    return torch.stack([a, a], dim=-2).contiguous()


@dataclass
class BatchWorkload:
    name: str
    lengths: np.ndarray          # int64 [nruns]
    couplings: np.ndarray        # float64 [nruns, 3]
    eps: float
    steps: int
    precision: int
    state: np.ndarray = field(repr=False)   # concatenated run states, each (5, 1, L, 2, 2) flattened
    meta: dict = field(default_factory=dict)

    def offsets(self) -> np.ndarray:
        """Element offset of each run inside the concatenated state (20 reals per site)."""
        return np.concatenate([[0], np.cumsum(self.lengths)[:-1]]) * 20

    def run_state(self, r: int) -> np.ndarray:
        o = int(self.offsets()[r])
        return self.state[o:o + 20 * int(self.lengths[r])].reshape(5, 1, int(self.lengths[r]), 2, 2)


def scattering_run(rng: np.random.Generator, L: int, eps: float) -> np.ndarray:
    """One seeded two-soliton scattering state of length L (the recipe of config1)."""
    rows = rng.choice([1, 2, 15], size=2, replace=False)
    kappa = rng.uniform(0.05, 0.3)
    n = int(round(kappa * L / (2 * np.pi)))
    rel = rng.uniform(0.0, 2 * np.pi)
    j = np.arange(L, dtype=np.float64)
    p_lat = 2 * np.pi * n / L
    s1 = bright_soliton(eps * (j - L / 4), int(rows[0]), CONFIG0_G)
    s2 = bright_soliton(eps * (j - 3 * L / 4), int(rows[1]), CONFIG0_G)
    return s1 * np.exp(1j * p_lat * j)[None, :] + s2 * np.exp(-1j * p_lat * j + 1j * rel)[None, :]


def config3(seed: int = 1910, nruns: int = 256, lmin: int = 2048, lmax: int = 65536,
            eps: float = 0.1, steps: int = 10000, dtype=np.float32) -> BatchWorkload:
    """Batched 1D scattering: nruns independent runs, L log-uniform in [lmin, lmax], each with
    its own seeded soliton pair (config1 recipe) and couplings g0 = 1, g1, g2 ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    lengths = np.exp(rng.uniform(np.log(lmin), np.log(lmax), size=nruns)).astype(np.int64)
    couplings = np.column_stack([np.ones(nruns), rng.uniform(-1, 1, nruns), rng.uniform(-1, 1, nruns)])
    parts = [boson_to_state(scattering_run(rng, int(L), eps), eps, dtype=dtype).ravel() for L in lengths]
    return BatchWorkload("1d-batched-scattering-%druns" % nruns, lengths, couplings, eps, steps,
                         32 if dtype == np.float32 else 64, np.concatenate(parts))


def batch2d(seed: int = 1912, nruns: int = 128, eps: float = 0.1, steps: int = 2000,
            dtype=np.float32) -> BatchWorkload:
    """Batched 2D vortex scattering: nruns independent runs of uneven size, nx = 32 k with k
    uniform in 2..16 (64 .. 512 columns), ny log-uniform in [64, 512]; each run holds the config 2
    dipole pair (variant a, cores nx / 4 apart, seeded integer kicks) at couplings g0 = 1 and
    g1, g2 uniform in [0.05, 0.5] x [0.5, 1.5] (the regime of the paper's 2D runs).  The state is
    the concatenation of the runs' 2D states; `meta["heights"]` holds each run's ny."""
    rng = np.random.default_rng(seed)
    nx = 32 * rng.integers(2, 17, size=nruns)
    ny = np.exp(rng.uniform(np.log(64), np.log(512), size=nruns)).astype(np.int64)
    couplings = np.column_stack([np.ones(nruns), rng.uniform(0.05, 0.5, nruns), rng.uniform(0.5, 1.5, nruns)])
    parts = []
    for r in range(nruns):
        g = tuple(couplings[r])
        psi = np.zeros((5, int(ny[r]), int(nx[r])), dtype=np.complex128)
        for k, mf in enumerate((2, -2)):
            kick = tuple(int(v) for v in rng.integers(-2, 3, size=2))
            psi[2 - mf] = vortex_dipole(int(nx[r]), int(ny[r]), eps, mf, CONFIG2_G, separation=nx[r] / 4.0,
                                        winding=+1 if k == 0 else -1, kick=kick)
        parts.append(boson_to_state(psi, eps, dtype=dtype).ravel())
    w = BatchWorkload("2d-batched-vortex-scattering-%druns" % nruns, nx.astype(np.int64), couplings, eps, steps,
                      32 if dtype == np.float32 else 64, np.concatenate(parts))
    w.meta["heights"] = ny.astype(np.int64)
    return w


# --------------------------------------------------------------------------- accuracy records
#
# Named workloads of the accuracy record: the FP64 oracle's results for them are stored under
# tests/golden/ (written by scripts there that call only the oracle), and the library's paths
# are run on the same inputs and compared.

LONG_HORIZON = ("config1_g_integrable_set", "config1_g_nonintegrable_set", "config2_512")
PERTURBATION = 1e-13


def long_horizon_workload(name):
    """(ndim, nx, ny, couplings, steps, checkpoint interval, FP64 initial state) of a long run:
    config 1 at full size and step count under each coupling set, and the config 2 recipe on a
    512^2 lattice for config 2's 5000 steps."""
    if name == "config1_g_integrable_set":       # the profiles' couplings (1, -0.5, 0.2)
        w = config1(L=16384, precision=64)
        return 1, 16384, 1, w.g, 20000, 1000, np.ascontiguousarray(w.state, dtype=np.float64)
    if name == "config1_g_nonintegrable_set":    # (1, 0.8, -0.6)
        w = config1(L=16384, precision=64, couplings=(1.0, 0.8, -0.6))
        return 1, 16384, 1, w.g, 20000, 1000, np.ascontiguousarray(w.state, dtype=np.float64)
    if name == "config2_512":
        w = config2(n=512, dtype=np.float64)
        return 2, 512, 512, w.g, 5000, 500, np.ascontiguousarray(w.state, dtype=np.float64)
    raise KeyError(name)


def perturbed(x0, rel=PERTURBATION, seed=2019):
    """x0 (1 + rel xi), xi seeded standard normal: a rounding-sized change of the initial state."""
    rng = np.random.default_rng(seed)
    return x0 * (1.0 + rel * rng.standard_normal(x0.shape))


def path_accuracy_workloads():
    """The short runs behind each timed path's accuracy statement (FP64 inputs): name ->
    dict(kind, steps, and the workload)."""
    return {
        "config0": {"kind": "lattice", "steps": 2000, "w": config0()},
        "interleaved": {"kind": "lattice", "steps": 100, "w": config2(n=128, dtype=np.float64),
                        "interleave": 1},
        "batch1d": {"kind": "batch", "steps": 500, "w": config3(nruns=6, lmin=512, lmax=2048, dtype=np.float64)},
        "batch2d": {"kind": "batch", "steps": 100, "w": batch2d(nruns=4, dtype=np.float64)},
        "adjoint": {"kind": "adjoint", "steps": 100, "w": config4(n=64, separation=20, dtype=np.float64),
                    "cotangent_seed": 1911},
    }


def adjoint_cotangent(shape, seed):
    """The seeded cotangent w of the adjoint accuracy run: L = <w, x_n>."""
    return np.random.default_rng(seed).standard_normal(shape)
