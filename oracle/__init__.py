"""Plain FP64 CPU oracle of the spin-2 BEC QLGA (arXiv:1907.12834).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline / reference leg of ``bench.py``; the library never imports it.  The arithmetic
lives in ``qlga_oracle.c`` (plain C, FP64, one operator at a time, U from a Hermitian
eigendecomposition); this module only compiles it with gcc and marshals numpy arrays.

State arrays are float64 of shape (5, ny, nx, 2, 2): level m = +2..-2, y, x, qubit (a, b),
(re, im) -- the library's data format.

Parity status of each function (what pins it; see tests/test_oracle_pins.py):
  potential_matrix  pinned: every Table I row is an eigenvector with eigenvalue E.
  expm / heig       pinned: scipy.linalg.expm, reconstruction and unitarity.
  apply_potential   pinned: uniform Thomas-Fermi state gains exactly exp(-i E delta).
  apply_kinetic     pinned: plane-wave Fourier symbol of the block product, the
                    -i p^2 + O(p^4) expansion of Sec. VII.B, dense brute force.
  step              pinned: dense brute-force operator product on tiny lattices, bright
                    soliton stationarity and drift velocity 2p (Sec. III/IV).
  observables       pinned: Table II characteristics, closed-form sums, brute force.
  fields            pinned: Table II characteristics per site, plane-wave velocity (zero
                    vorticity), total vorticity of a vortex / antivortex (+-2 pi), colour norm.
  frechet_exp       pinned: block-triangular exponential exp([[A, E], [0, A]]) (scipy).
  vjp_kinetic       pinned: dot-product identity <K v, w> = <v, K^dagger w>, K^dagger K = 1.
  vjp_potential /   pinned: central finite differences of the (pinned) forward operators in
  vjp_step / run    random directions, coupling derivatives by finite differences in g.
  step_long_double  not a pin: the same source built in long double, which bounds the FP64
                    oracle's own rounding (tests/test_oracle_precision.py).

Adjoint cotangents: for a real loss L the cotangent array has the state's shape and holds
dL/d(each real component); dL = sum(cot * dx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qlga_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

N_OBS = 15


class OracleCfg(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("nx", ctypes.c_long),
        ("ny", ctypes.c_long),
        ("g0", ctypes.c_double),
        ("g1", ctypes.c_double),
        ("g2", ctypes.c_double),
        ("interleave", ctypes.c_int),
        ("kinetic_variant", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile qlga_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_LIB_LD = os.path.join(_HERE, "liboracle_ld.so")

# Appended to the long-double source: a float64 state in, nsteps in extended precision, one
# rounding to float64 on the way out.
_LD_ENTRY = r"""
int oracle_step_from_double(const double* in, double* out, const oracle_cfg_f64* c, long nsteps,
                            int nthreads) {
    const long n = 5 * c->nx * c->ny * 4;
    long double* st = (long double*)malloc(sizeof(long double) * (size_t)n);
    if (!st) return 2;
    for (long i = 0; i < n; ++i) st[i] = in[i];
    oracle_cfg cfg = {c->ndim, c->nx, c->ny, c->g0, c->g1, c->g2, c->interleave, c->kinetic_variant};
    const int rc = oracle_step(st, &cfg, nsteps, nthreads);
    for (long i = 0; i < n; ++i) out[i] = (double)st[i];
    free(st);
    return rc;
}
"""


def long_double_source(src_text: str = None) -> str:
    """The oracle's C source with every `double` made `long double` and the math calls made
    type-generic (<tgmath.h>), plus the entry point oracle_step_from_double.  It is the same
    algorithm evaluated with a longer significand (64 bits on x86-64, 113 on aarch64), used only
    to measure how far the FP64 oracle's own rounding carries it.  Constants the source computes
    from double arguments (sqrt(1.5) of the spin matrices) stay the FP64 values, so both builds
    evaluate the same discrete operator."""
    import re

    src = open(_SRC).read() if src_text is None else src_text
    head = "#include <complex.h>\n#include <math.h>\n"
    if head not in src or "long double" in src:
        raise ValueError("unexpected oracle source layout")
    src = src.replace(head, "#include <tgmath.h>\n", 1)
    cfg_f64 = src[src.index("typedef struct oracle_cfg {"):src.index("} oracle_cfg;") + len("} oracle_cfg;")]
    cfg_f64 = cfg_f64.replace("oracle_cfg {", "oracle_cfg_f64 {").replace("} oracle_cfg;", "} oracle_cfg_f64;")
    src = re.sub(r"\bdouble\b", "long double", src)
    return src + "\n" + cfg_f64 + "\n" + _LD_ENTRY


def build_long_double(force: bool = False) -> str:
    """Compile long_double_source() into liboracle_ld.so (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB_LD) and os.path.getmtime(_LIB_LD) >= os.path.getmtime(_SRC):
        return _LIB_LD
    tmp = _LIB_LD + ".%d.tmp" % os.getpid()
    src = tmp + ".c"
    with open(src, "w") as f:
        f.write(long_double_source())
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"],
                   check=True)
    os.remove(src)
    os.replace(tmp, _LIB_LD)
    return _LIB_LD


def step_long_double(state: np.ndarray, cfg: OracleCfg, nsteps: int, nthreads: int = 0) -> np.ndarray:
    """A copy of `state` advanced nsteps QLGA steps by the long-double build of the oracle."""
    _check_state(state, cfg)
    lib = ctypes.CDLL(build_long_double())
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_step_from_double.argtypes = [dp, dp, ctypes.POINTER(OracleCfg), ctypes.c_long, ctypes.c_int]
    lib.oracle_step_from_double.restype = ctypes.c_int
    out = np.empty_like(state)
    if lib.oracle_step_from_double(_dptr(state), _dptr(out), ctypes.byref(cfg), int(nsteps), int(nthreads)):
        raise ValueError("oracle_step_from_double rejected its arguments")
    return out


def compile_source(src_text: str, out_path: str) -> str:
    """Compile a (possibly edited) copy of the oracle source; used by the mutation tests
    that check the pins catch a planted mistake."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", out_path,
                    src, "-lm"], check=True)
    return out_path


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_cfg(ndim, nx, ny, g0, g1, g2, interleave=0, kinetic_variant=0) -> OracleCfg:
    return OracleCfg(int(ndim), int(nx), int(ny), float(g0), float(g1), float(g2),
                     int(interleave), int(kinetic_variant))


def _check_state(state: np.ndarray, cfg: OracleCfg) -> np.ndarray:
    if state.dtype != np.float64 or not state.flags.c_contiguous:
        raise TypeError("oracle state must be a C-contiguous float64 array")
    if state.shape != (5, cfg.ny, cfg.nx, 2, 2):
        raise ValueError("oracle state shape %r does not match cfg" % (state.shape,))
    return state


OBS_NAMES = ("norm_qubit", "norm_boson", "pop_p2", "pop_p1", "pop_0", "pop_m1", "pop_m2",
             "magnetisation", "energy", "singlet_re", "singlet_im", "theta2_sum", "rho2_sum",
             "overlap_re", "overlap_im")


def _mat_to_buf(M: np.ndarray) -> np.ndarray:
    M = np.asarray(M, dtype=np.complex128).reshape(25)
    return np.ascontiguousarray(np.column_stack([M.real, M.imag]).ravel())


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        cp = ctypes.POINTER(OracleCfg)
        lib.oracle_step.argtypes = [dp, cp, ctypes.c_long, ctypes.c_int]
        lib.oracle_apply_potential.argtypes = [dp, cp, ctypes.c_double, ctypes.c_int]
        lib.oracle_apply_kinetic.argtypes = [dp, cp, ctypes.c_int]
        lib.oracle_apply_operator.argtypes = [dp, cp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int]
        lib.oracle_observables.argtypes = [dp, dp, cp, dp]
        lib.oracle_potential_matrix.argtypes = [dp, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, dp]
        lib.oracle_heig.argtypes = [dp, dp, dp]
        lib.oracle_expm.argtypes = [dp, ctypes.c_double, dp]
        lib.oracle_max_threads.argtypes = []
        lib.oracle_fields.argtypes = [dp, cp, dp]
        lib.oracle_vjp_potential.argtypes = [dp, dp, cp, ctypes.c_double, dp, ctypes.c_int]
        lib.oracle_vjp_kinetic.argtypes = [dp, cp, ctypes.c_int]
        lib.oracle_vjp_step.argtypes = [dp, dp, cp, dp, ctypes.c_int]
        lib.oracle_vjp_run.argtypes = [dp, ctypes.c_long, dp, cp, dp, ctypes.c_int]
        lib.oracle_frechet_exp.argtypes = [dp, ctypes.c_double, dp, dp]
        for name in ("oracle_step", "oracle_apply_potential", "oracle_apply_kinetic",
                     "oracle_apply_operator", "oracle_observables", "oracle_potential_matrix",
                     "oracle_heig", "oracle_expm", "oracle_max_threads", "oracle_fields",
                     "oracle_vjp_potential", "oracle_vjp_kinetic", "oracle_vjp_step",
                     "oracle_vjp_run", "oracle_frechet_exp"):
            getattr(lib, name).restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())

    def step(self, state: np.ndarray, cfg: OracleCfg, nsteps: int, nthreads: int = 0):
        """Advance `state` in place by nsteps QLGA time steps."""
        _check_state(state, cfg)
        if self.lib.oracle_step(_dptr(state), ctypes.byref(cfg), int(nsteps), int(nthreads)):
            raise ValueError("oracle_step rejected its arguments")
        return state

    def apply_potential(self, state, cfg, delta=1.0, nthreads=0):
        _check_state(state, cfg)
        if self.lib.oracle_apply_potential(_dptr(state), ctypes.byref(cfg), float(delta),
                                           int(nthreads)):
            raise ValueError("bad arguments")
        return state

    def apply_kinetic(self, state, cfg, nthreads=0):
        _check_state(state, cfg)
        if self.lib.oracle_apply_kinetic(_dptr(state), ctypes.byref(cfg), int(nthreads)):
            raise ValueError("bad arguments")
        return state

    def apply_operator(self, state, cfg, which, axis=0, q=0, direction=1):
        """which: 0 first collide, 1 second collide, 2 stream qubit q along axis."""
        _check_state(state, cfg)
        if self.lib.oracle_apply_operator(_dptr(state), ctypes.byref(cfg), int(which),
                                          int(axis), int(q), int(direction)):
            raise ValueError("bad arguments")
        return state

    def observables(self, state, cfg, ref=None) -> dict:
        _check_state(state, cfg)
        out = np.zeros(N_OBS)
        refp = None
        if ref is not None:
            _check_state(ref, cfg)
            refp = _dptr(ref)
        if self.lib.oracle_observables(_dptr(state), refp, ctypes.byref(cfg), _dptr(out)):
            raise ValueError("bad arguments")
        d = dict(zip(OBS_NAMES, out.tolist()))
        d["pop"] = out[2:7].copy()
        d["singlet_fraction"] = d["theta2_sum"] / d["rho2_sum"] if d["rho2_sum"] > 0 else 0.0
        return d

    def fields(self, state, cfg) -> np.ndarray:
        """Per-site fields, shape (11, ny, nx): F_par, F_perp, |A00|, r, g, b, vorticity m=+2..-2."""
        _check_state(state, cfg)
        out = np.zeros((11, cfg.ny, cfg.nx))
        if self.lib.oracle_fields(_dptr(state), ctypes.byref(cfg), _dptr(out)):
            raise ValueError("bad arguments")
        return out

    def potential_matrix(self, psi, g0, g1, g2) -> np.ndarray:
        """V(psi) as a 5x5 complex matrix for one site's boson 5-vector psi (m = +2..-2)."""
        psi = np.asarray(psi, dtype=np.complex128)
        p = np.ascontiguousarray(np.column_stack([psi.real, psi.imag]).ravel())
        out = np.zeros(50)
        self.lib.oracle_potential_matrix(_dptr(p), float(g0), float(g1), float(g2), _dptr(out))
        return (out[0::2] + 1j * out[1::2]).reshape(5, 5)

    def heig(self, V):
        lam = np.zeros(5)
        Q = np.zeros(50)
        self.lib.oracle_heig(_dptr(_mat_to_buf(V)), _dptr(lam), _dptr(Q))
        return lam, (Q[0::2] + 1j * Q[1::2]).reshape(5, 5)

    def expm(self, V, delta: float) -> np.ndarray:
        """exp(-i delta V) of a Hermitian 5x5 matrix."""
        U = np.zeros(50)
        self.lib.oracle_expm(_dptr(_mat_to_buf(V)), float(delta), _dptr(U))
        return (U[0::2] + 1j * U[1::2]).reshape(5, 5)

    # ------------------------------------------------------------ adjoint
    def vjp_potential(self, state, cot, cfg, delta=1.0, nthreads=0):
        """cot (cotangent of U(x) x) -> cotangent of x, in place; returns dL/d(g0, g1, g2)."""
        _check_state(state, cfg)
        _check_state(cot, cfg)
        d = np.zeros(3)
        if self.lib.oracle_vjp_potential(_dptr(state), _dptr(cot), ctypes.byref(cfg), float(delta),
                                         _dptr(d), int(nthreads)):
            raise ValueError("bad arguments")
        return d

    def vjp_kinetic(self, field, cfg, nthreads=0):
        """field <- K^dagger field, in place."""
        _check_state(field, cfg)
        if self.lib.oracle_vjp_kinetic(_dptr(field), ctypes.byref(cfg), int(nthreads)):
            raise ValueError("bad arguments")
        return field

    def vjp_step(self, state, cot, cfg, nthreads=0):
        """cot (cotangent of step(x)) -> cotangent of x, in place; returns dL/d(g0, g1, g2)."""
        _check_state(state, cfg)
        _check_state(cot, cfg)
        d = np.zeros(3)
        rc = self.lib.oracle_vjp_step(_dptr(state), _dptr(cot), ctypes.byref(cfg), _dptr(d), int(nthreads))
        if rc:
            raise ValueError("oracle_vjp_step rejected its arguments (%d)" % rc)
        return d

    def vjp_run(self, x0, nsteps, cot, cfg, nthreads=0):
        """Gradient through nsteps plain steps from x0: cot (cotangent of the final state) ->
        cotangent of x0, in place; returns dL/d(g0, g1, g2)."""
        _check_state(x0, cfg)
        _check_state(cot, cfg)
        d = np.zeros(3)
        rc = self.lib.oracle_vjp_run(_dptr(x0), int(nsteps), _dptr(cot), ctypes.byref(cfg), _dptr(d),
                                     int(nthreads))
        if rc:
            raise ValueError("oracle_vjp_run rejected its arguments (%d)" % rc)
        return d

    def frechet_exp(self, V, delta, E) -> np.ndarray:
        """L(-i delta V, E): the Frechet derivative of exp at -i delta V in direction E."""
        out = np.zeros(50)
        self.lib.oracle_frechet_exp(_dptr(_mat_to_buf(V)), float(delta), _dptr(_mat_to_buf(E)), _dptr(out))
        return (out[0::2] + 1j * out[1::2]).reshape(5, 5)


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def max_threads():
    return default().max_threads()


def step(state, cfg, nsteps, nthreads=0):
    return default().step(state, cfg, nsteps, nthreads)


def apply_potential(state, cfg, delta=1.0, nthreads=0):
    return default().apply_potential(state, cfg, delta, nthreads)


def apply_kinetic(state, cfg, nthreads=0):
    return default().apply_kinetic(state, cfg, nthreads)


def apply_operator(state, cfg, which, axis=0, q=0, direction=1):
    return default().apply_operator(state, cfg, which, axis, q, direction)


def observables(state, cfg, ref=None):
    return default().observables(state, cfg, ref)


def potential_matrix(psi, g0, g1, g2):
    return default().potential_matrix(psi, g0, g1, g2)


def fields(state, cfg):
    return default().fields(state, cfg)


def heig(V):
    return default().heig(V)


def expm(V, delta):
    return default().expm(V, delta)


def vjp_potential(state, cot, cfg, delta=1.0, nthreads=0):
    return default().vjp_potential(state, cot, cfg, delta, nthreads)


def vjp_kinetic(field, cfg, nthreads=0):
    return default().vjp_kinetic(field, cfg, nthreads)


def vjp_step(state, cot, cfg, nthreads=0):
    return default().vjp_step(state, cot, cfg, nthreads)


def vjp_run(x0, nsteps, cot, cfg, nthreads=0):
    return default().vjp_run(x0, nsteps, cot, cfg, nthreads)


def frechet_exp(V, delta, E):
    return default().frechet_exp(V, delta, E)


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
