"""Python binding of the C ABI in include/qlga.h (argument marshalling only).

Every step of the QLGA runs in the CUDA kernels of ``libqlga.so``.  PyTorch supplies device
memory (``torch.empty`` buffers handed to ``qlga_create_external``) and the CUDA stream.  If the
library is missing this module raises; there is no CPU fallback.

Low level: the C entry points under the same names (``qlga_create``, ``qlga_step`` ...).
High level: :class:`Lattice`, which owns a handle and its torch buffers.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

QLGA_OK, QLGA_ERR_INVALID_ARG, QLGA_ERR_OOM, QLGA_ERR_CUDA, QLGA_ERR_TIMEOUT, \
    QLGA_ERR_NOT_FINITE, QLGA_ERR_UNSUPPORTED = range(7)
QLGA_HOST, QLGA_DEVICE = 0, 1
QLGA_KINETIC_K1, QLGA_KINETIC_K2 = 0, 1
QLGA_STEP2D_AUTO, QLGA_STEP2D_FUSED, QLGA_STEP2D_TWO_PASS = 0, 1, 2


class QlgaConfig(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("g0", ctypes.c_double), ("g1", ctypes.c_double), ("g2", ctypes.c_double),
                ("epsilon", ctypes.c_double), ("interleave", ctypes.c_int32),
                ("kinetic_variant", ctypes.c_int32)]


class QlgaObs(ctypes.Structure):
    _fields_ = [("norm_qubit", ctypes.c_double), ("norm_boson", ctypes.c_double),
                ("pop", ctypes.c_double * 5), ("magnetisation", ctypes.c_double),
                ("energy", ctypes.c_double), ("singlet_re", ctypes.c_double),
                ("singlet_im", ctypes.c_double), ("singlet_fraction", ctypes.c_double),
                ("overlap_re", ctypes.c_double), ("overlap_im", ctypes.c_double),
                ("step", ctypes.c_int64)]


class QlgaBatchConfig(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("nruns", ctypes.c_int32),
                ("lengths", ctypes.POINTER(ctypes.c_int64)),
                ("couplings", ctypes.POINTER(ctypes.c_double)),
                ("epsilon", ctypes.c_double), ("kinetic_variant", ctypes.c_int32),
                ("use_graph", ctypes.c_int32),
                ("heights", ctypes.POINTER(ctypes.c_int64))]


class QlgaError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__("%s failed: %s (%s)" % (where, _status_names.get(status, status), message))
        self.status = status


_status_names = {0: "QLGA_OK", 1: "QLGA_ERR_INVALID_ARG", 2: "QLGA_ERR_OOM", 3: "QLGA_ERR_CUDA",
                 4: "QLGA_ERR_TIMEOUT", 5: "QLGA_ERR_NOT_FINITE", 6: "QLGA_ERR_UNSUPPORTED"}

_lib = None
_VP = ctypes.c_void_p
_CFG = ctypes.POINTER(QlgaConfig)
_H = ctypes.c_void_p

_SIGNATURES = {
    "qlga_state_bytes": [_CFG, ctypes.POINTER(ctypes.c_size_t)],
    "qlga_workspace_bytes": [_CFG, ctypes.POINTER(ctypes.c_size_t)],
    "qlga_create": [_CFG, _VP, ctypes.POINTER(_H)],
    "qlga_create_external": [_CFG, _VP, _VP, _VP, _VP, ctypes.c_size_t, ctypes.POINTER(_H)],
    "qlga_load_state": [_H, _VP, ctypes.c_int],
    "qlga_load_boson": [_H, _VP, ctypes.c_int],
    "qlga_get_state": [_H, _VP, ctypes.c_int],
    "qlga_step": [_H, ctypes.c_int64],
    "qlga_apply_potential": [_H, ctypes.c_double],
    "qlga_apply_kinetic": [_H],
    "qlga_observables": [_H, _VP, ctypes.POINTER(QlgaObs)],
    "qlga_synchronize": [_H],
    "qlga_launch_count": [_H, ctypes.POINTER(ctypes.c_int64)],
    "qlga_set_graph_steps": [_H, ctypes.c_int32],
    "qlga_set_step2d_mode": [_H, ctypes.c_int32],
    "qlga_get_step2d_kernel": [_H, ctypes.POINTER(ctypes.c_int32)],
    "qlga_observables_noalloc": [_CFG, _VP, _VP, _VP, ctypes.POINTER(QlgaObs)],
    "qlga_fields": [_H, _VP, ctypes.c_int],
    "qlga_copy_rows": [_H, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int],
    "qlga_objective": [_H, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _VP],
    "qlga_exchange_rows": [_H, ctypes.c_int64, _H, ctypes.c_int64, ctypes.c_int64],
    "qlga_observable_sums": [_H, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_double)],
    "qlga_obs_from_sums": [ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.POINTER(QlgaObs)],
    "qlga_batch_state_bytes": [ctypes.POINTER(QlgaBatchConfig), ctypes.POINTER(ctypes.c_size_t)],
    "qlga_batch_create": [ctypes.POINTER(QlgaBatchConfig), _VP, ctypes.POINTER(_H)],
    "qlga_batch_load_state": [_H, _VP, ctypes.c_int],
    "qlga_batch_get_state": [_H, _VP, ctypes.c_int],
    "qlga_batch_step": [_H, ctypes.c_int64],
    "qlga_batch_observables": [_H, ctypes.POINTER(QlgaObs)],
    "qlga_batch_info": [_H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int32)],
    "qlga_batch_set_shape": [_H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
    "qlga_set_1d_shape": [_H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
    "qlga_get_1d_shape": [_H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_int32)],
    "qlga_batch_destroy": [_H],
    "qlga_destroy": [_H],
    "qlga_adjoint_workspace_bytes": [_CFG, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)],
    "qlga_adjoint_forward": [_H, _VP, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_size_t],
    "qlga_adjoint_backward": [_H, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_size_t, _VP,
                              ctypes.POINTER(ctypes.c_double)],
    "qlga_adjoint_run": [_H, _VP, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_size_t, _VP,
                         ctypes.POINTER(ctypes.c_double)],
    "qlga_adjoint_step": [_H, _VP, _VP, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)],
}


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libqlga.so (building it with nvcc if absent and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libqlga.so is not built (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, argtypes in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = argtypes
        fn.restype = ctypes.c_int
    lib.qlga_status_string.argtypes = [ctypes.c_int]
    lib.qlga_status_string.restype = ctypes.c_char_p
    lib.qlga_last_error.argtypes = []
    lib.qlga_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def header_symbols() -> list:
    """Entry points declared in include/qlga.h."""
    hdr = os.path.join(_build.ROOT, "include", "qlga.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:qlga_status|const char\*)\s+(qlga_\w+)\s*\(", text, re.M)))


def _check(status: int, where: str):
    if status != QLGA_OK:
        lib = load_library()
        raise QlgaError(status, where, lib.qlga_last_error().decode())


# ------------------------------------------------------------------ C entry points, same names

def make_config(ndim, nx, ny=1, precision=64, g=(1.0, 0.0, 0.0), epsilon=0.1, interleave=0,
                kinetic_variant=0) -> QlgaConfig:
    return QlgaConfig(int(ndim), int(precision), int(nx), int(ny), float(g[0]), float(g[1]),
                      float(g[2]), float(epsilon), int(interleave), int(kinetic_variant))


def qlga_state_bytes(cfg: QlgaConfig) -> int:
    out = ctypes.c_size_t()
    _check(load_library().qlga_state_bytes(ctypes.byref(cfg), ctypes.byref(out)), "qlga_state_bytes")
    return out.value


def qlga_workspace_bytes(cfg: QlgaConfig) -> int:
    out = ctypes.c_size_t()
    _check(load_library().qlga_workspace_bytes(ctypes.byref(cfg), ctypes.byref(out)),
           "qlga_workspace_bytes")
    return out.value


def qlga_create(cfg: QlgaConfig, stream: int = 0) -> int:
    h = _H()
    _check(load_library().qlga_create(ctypes.byref(cfg), _VP(stream), ctypes.byref(h)), "qlga_create")
    return h.value


def qlga_create_external(cfg, stream, state0, state1, workspace, workspace_bytes) -> int:
    h = _H()
    _check(load_library().qlga_create_external(ctypes.byref(cfg), _VP(stream), _VP(state0),
                                               _VP(state1), _VP(workspace),
                                               ctypes.c_size_t(workspace_bytes), ctypes.byref(h)),
           "qlga_create_external")
    return h.value


def qlga_load_state(h: int, ptr: int, where: int):
    _check(load_library().qlga_load_state(_H(h), _VP(ptr), int(where)), "qlga_load_state")


def qlga_load_boson(h: int, ptr: int, where: int):
    _check(load_library().qlga_load_boson(_H(h), _VP(ptr), int(where)), "qlga_load_boson")


def qlga_get_state(h: int, ptr: int, where: int):
    _check(load_library().qlga_get_state(_H(h), _VP(ptr), int(where)), "qlga_get_state")


def qlga_step(h: int, n: int):
    _check(load_library().qlga_step(_H(h), ctypes.c_int64(int(n))), "qlga_step")


def qlga_apply_potential(h: int, delta: float):
    _check(load_library().qlga_apply_potential(_H(h), ctypes.c_double(delta)), "qlga_apply_potential")


def qlga_apply_kinetic(h: int):
    _check(load_library().qlga_apply_kinetic(_H(h)), "qlga_apply_kinetic")


def qlga_observables(h: int, ref_ptr: int = 0) -> QlgaObs:
    out = QlgaObs()
    _check(load_library().qlga_observables(_H(h), _VP(ref_ptr or None), ctypes.byref(out)),
           "qlga_observables")
    return out


def qlga_observables_noalloc(cfg: QlgaConfig, state_ptr: int, ref_ptr: int = 0,
                             stream: int = 0) -> QlgaObs:
    """Observables of a device state with no device allocation (static library scratch)."""
    out = QlgaObs()
    _check(load_library().qlga_observables_noalloc(ctypes.byref(cfg), _VP(state_ptr),
                                                   _VP(ref_ptr or None), _VP(stream or None),
                                                   ctypes.byref(out)),
           "qlga_observables_noalloc")
    return out


def _dbl3(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def qlga_objective(h: int, x_ptr: int, level: int, g, weights=None, cot_ptr: int = 0):
    """(values[3], dg[3] or None) of qlga_objective; the cotangent goes to cot_ptr if given."""
    ga, gp = _dbl3(g)
    vals = np.zeros(3)
    dg = np.zeros(3) if weights is not None else None
    wa, wp = _dbl3(weights) if weights is not None else (None, None)
    _check(load_library().qlga_objective(_H(h), _VP(x_ptr), int(level), gp, wp,
                                         vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         dg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if dg is not None else None,
                                         _VP(cot_ptr or None)),
           "qlga_objective")
    return vals, dg


QLGA_ROWS_OUT, QLGA_ROWS_IN = 0, 1


def qlga_copy_rows(h: int, y0: int, nrows: int, ptr: int, direction: int):
    _check(load_library().qlga_copy_rows(_H(h), int(y0), int(nrows), _VP(ptr), int(direction)),
           "qlga_copy_rows")


def qlga_exchange_rows(src: int, ysrc: int, dst: int, ydst: int, nrows: int):
    _check(load_library().qlga_exchange_rows(_H(src), int(ysrc), _H(dst), int(ydst), int(nrows)),
           "qlga_exchange_rows")


def qlga_observable_sums(h: int, y0: int, y1: int, ref_ptr: int = 0) -> np.ndarray:
    out = np.zeros(14, dtype=np.float64)
    _check(load_library().qlga_observable_sums(_H(h), int(y0), int(y1), _VP(ref_ptr or None),
                                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "qlga_observable_sums")
    return out


def qlga_obs_from_sums(sums, step: int = 0) -> QlgaObs:
    a = np.ascontiguousarray(sums, dtype=np.float64)
    if a.shape != (14,):
        raise ValueError("sums must hold 14 values")
    out = QlgaObs()
    _check(load_library().qlga_obs_from_sums(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(step),
                                             ctypes.byref(out)),
           "qlga_obs_from_sums")
    return out


def qlga_fields(h: int, ptr: int, where: int):
    _check(load_library().qlga_fields(_H(h), _VP(ptr), int(where)), "qlga_fields")


def qlga_launch_count(h: int) -> int:
    out = ctypes.c_int64()
    _check(load_library().qlga_launch_count(_H(h), ctypes.byref(out)), "qlga_launch_count")
    return out.value


def qlga_set_graph_steps(h: int, steps: int):
    _check(load_library().qlga_set_graph_steps(_H(h), ctypes.c_int32(int(steps))), "qlga_set_graph_steps")


def qlga_set_step2d_mode(h: int, mode: int):
    _check(load_library().qlga_set_step2d_mode(_H(h), ctypes.c_int32(int(mode))), "qlga_set_step2d_mode")


def qlga_get_step2d_kernel(h: int) -> int:
    out = ctypes.c_int32()
    _check(load_library().qlga_get_step2d_kernel(_H(h), ctypes.byref(out)), "qlga_get_step2d_kernel")
    return out.value


def qlga_synchronize(h: int):
    _check(load_library().qlga_synchronize(_H(h)), "qlga_synchronize")


def qlga_destroy(h: int):
    _check(load_library().qlga_destroy(_H(h)), "qlga_destroy")


def qlga_adjoint_workspace_bytes(cfg: QlgaConfig, nsteps: int, checkpoint_every: int) -> int:
    out = ctypes.c_size_t()
    _check(load_library().qlga_adjoint_workspace_bytes(ctypes.byref(cfg), ctypes.c_int64(int(nsteps)),
                                                       ctypes.c_int64(int(checkpoint_every)),
                                                       ctypes.byref(out)), "qlga_adjoint_workspace_bytes")
    return out.value


def qlga_adjoint_forward(h, x0_ptr, nsteps, checkpoint_every, ws_ptr, ws_bytes):
    _check(load_library().qlga_adjoint_forward(_H(h), _VP(x0_ptr), ctypes.c_int64(int(nsteps)),
                                               ctypes.c_int64(int(checkpoint_every)), _VP(ws_ptr),
                                               ctypes.c_size_t(ws_bytes)), "qlga_adjoint_forward")


def qlga_adjoint_backward(h, nsteps, checkpoint_every, ws_ptr, ws_bytes, cot_ptr) -> np.ndarray:
    d = (ctypes.c_double * 3)()
    _check(load_library().qlga_adjoint_backward(_H(h), ctypes.c_int64(int(nsteps)),
                                                ctypes.c_int64(int(checkpoint_every)), _VP(ws_ptr),
                                                ctypes.c_size_t(ws_bytes), _VP(cot_ptr), d),
           "qlga_adjoint_backward")
    return np.array(list(d))


def qlga_adjoint_run(h, x0_ptr, nsteps, checkpoint_every, ws_ptr, ws_bytes, cot_ptr) -> np.ndarray:
    d = (ctypes.c_double * 3)()
    _check(load_library().qlga_adjoint_run(_H(h), _VP(x0_ptr), ctypes.c_int64(int(nsteps)),
                                           ctypes.c_int64(int(checkpoint_every)), _VP(ws_ptr),
                                           ctypes.c_size_t(ws_bytes), _VP(cot_ptr), d), "qlga_adjoint_run")
    return np.array(list(d))


def qlga_adjoint_step(h, x_ptr, cot_ptr, ws_ptr, ws_bytes) -> np.ndarray:
    d = (ctypes.c_double * 3)()
    _check(load_library().qlga_adjoint_step(_H(h), _VP(x_ptr), _VP(cot_ptr), _VP(ws_ptr),
                                            ctypes.c_size_t(ws_bytes), d), "qlga_adjoint_step")
    return np.array(list(d))


def qlga_status_string(status: int) -> str:
    return load_library().qlga_status_string(int(status)).decode()


def qlga_last_error() -> str:
    return load_library().qlga_last_error().decode()


def obs_to_dict(o: QlgaObs) -> dict:
    d = {k: getattr(o, k) for k, _ in QlgaObs._fields_ if k != "pop"}
    d["pop"] = np.array(list(o.pop))
    return d


# ------------------------------------------------------------------ buffer checks
#
# The library reads or writes the whole extent of a buffer through a raw pointer, so a buffer of
# the wrong size, type or device would be read or written past its end.  These checks run before
# every such call of the classes below (and are not asserts, which `python -O` removes).

def require_device_tensor(t, shape, dtype, device, what, writable=False):
    """Raise unless `t` is a CUDA tensor of `shape` and `dtype` on `device` (contiguous when the
    library writes into it)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError("%s must be %s of shape %s, got %s of shape %s"
                         % (what, dtype, tuple(shape), t.dtype, tuple(t.shape)))
    if t.device.index != device.index:
        raise ValueError("%s is on %s, the lattice on %s" % (what, t.device, device))
    if writable and not t.is_contiguous():
        raise ValueError("%s must be contiguous: the library writes into it" % what)
    return t


def require_host_array(a, shape, dtype, what, writable=False):
    """Raise unless `a` is a C-contiguous numpy array of `shape` and `dtype` (writeable when the
    library writes into it)."""
    if not isinstance(a, np.ndarray) or a.dtype != dtype or a.shape != tuple(shape):
        raise ValueError("%s must be a numpy array of %s and shape %s" % (what, np.dtype(dtype), tuple(shape)))
    if not a.flags.c_contiguous or (writable and not a.flags.writeable):
        raise ValueError("%s must be C-contiguous%s" % (what, " and writeable" if writable else ""))
    return a


# ------------------------------------------------------------------ high-level lattice

class Lattice:
    """A QLGA lattice on the current CUDA device, in torch-allocated device memory.

    ``state`` arrays use the library layout (5, ny, nx, 2, 2): level m = +2..-2, y, x,
    qubit (a, b), (re, im); float32 for precision 32, float64 for 64.
    """

    def __init__(self, ndim, nx, ny=1, precision=64, g=(1.0, 0.0, 0.0), epsilon=0.1,
                 interleave=0, kinetic_variant=0, stream=None, device=None):
        import torch
        self._torch = torch
        self.cfg = make_config(ndim, nx, ny, precision, g, epsilon, interleave, kinetic_variant)
        self.shape = (5, int(ny), int(nx), 2, 2)
        self.dtype = np.float32 if precision == 32 else np.float64
        self.tdtype = torch.float32 if precision == 32 else torch.float64
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        sb = qlga_state_bytes(self.cfg)
        wb = qlga_workspace_bytes(self.cfg)
        with torch.cuda.device(dev):
            # 256-byte aligned blocks from the caching allocator
            self._bufs = [torch.empty(sb + 256, dtype=torch.uint8, device=dev) for _ in range(2)]
            self._ws = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            ptrs = [self._aligned(b) for b in self._bufs]
            self.handle = qlga_create_external(self.cfg, self.stream.cuda_stream, ptrs[0], ptrs[1],
                                               self._aligned(self._ws), wb)
        self.state_bytes = sb

    @staticmethod
    def _aligned(t):
        p = t.data_ptr()
        return (p + 255) & ~255

    # -- state transfer
    def load_state(self, state):
        """Host numpy array or device torch tensor of the library layout."""
        torch = self._torch
        if isinstance(state, torch.Tensor):
            if not state.is_cuda:
                state = state.numpy()
            else:
                t = require_device_tensor(state, self.shape, self.tdtype, self.device, "state").contiguous()
                qlga_load_state(self.handle, t.data_ptr(), QLGA_DEVICE)
                return
        a = require_host_array(np.ascontiguousarray(state, dtype=self.dtype), self.shape, self.dtype, "state")
        qlga_load_state(self.handle, a.ctypes.data, QLGA_HOST)

    def load_boson(self, psi):
        """Physical boson field psi[5, ny, nx] (complex): a = b = epsilon psi / 2."""
        z = np.asarray(psi).reshape(5, self.shape[1], self.shape[2])
        a = np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1), dtype=self.dtype)
        qlga_load_boson(self.handle, a.ctypes.data, QLGA_HOST)

    def get_state(self, out=None):
        """Copy of the current state: numpy (host) by default, or into a device tensor."""
        torch = self._torch
        if out is not None and isinstance(out, torch.Tensor) and out.is_cuda:
            require_device_tensor(out, self.shape, self.tdtype, self.device, "out", writable=True)
            qlga_get_state(self.handle, out.data_ptr(), QLGA_DEVICE)
            return out
        if out is None:
            host = np.empty(self.shape, dtype=self.dtype)
        else:
            host = require_host_array(out, self.shape, self.dtype, "out", writable=True)
        qlga_get_state(self.handle, host.ctypes.data, QLGA_HOST)
        return host

    def device_state(self):
        t = self._torch.empty(self.shape, dtype=self.tdtype, device=self.device)
        qlga_get_state(self.handle, t.data_ptr(), QLGA_DEVICE)
        return t

    # -- time stepping
    def step(self, n=1):
        qlga_step(self.handle, n)

    def apply_potential(self, delta=1.0):
        qlga_apply_potential(self.handle, delta)

    def apply_kinetic(self):
        qlga_apply_kinetic(self.handle)

    def observables(self, ref=None) -> dict:
        ref_ptr = 0
        if ref is not None:
            ref = require_device_tensor(ref, self.shape, self.tdtype, self.device, "ref").contiguous()
            ref_ptr = ref.data_ptr()
        return obs_to_dict(qlga_observables(self.handle, ref_ptr))

    def copy_rows_out(self, y0, nrows, out=None):
        """Rows [y0, y0 + nrows) of the current buffer, as held, into a device tensor of
        5 * nrows * nx sites (float32 x4 or float64 x4 per site)."""
        torch = self._torch
        shape = (5, int(nrows), self.shape[2], 4)
        if out is None:
            out = torch.empty(shape, dtype=self.tdtype, device=self.device)
        out = require_device_tensor(out, shape, self.tdtype, self.device, "rows", writable=True)
        qlga_copy_rows(self.handle, y0, nrows, out.data_ptr(), QLGA_ROWS_OUT)
        return out

    def copy_rows_in(self, y0, rows):
        """Write rows [y0, y0 + rows.shape[1]) of the current buffer from a device tensor made
        by copy_rows_out on a handle of the same nx and precision."""
        nrows = int(rows.shape[1])
        rows = require_device_tensor(rows, (5, nrows, self.shape[2], 4), self.tdtype, self.device,
                                     "rows").contiguous()
        qlga_copy_rows(self.handle, y0, nrows, rows.data_ptr(), QLGA_ROWS_IN)

    def observable_sums(self, y0=0, y1=None, ref=None) -> np.ndarray:
        """The 14 FP64 sums behind observables() over rows [y0, y1)."""
        ref_ptr = 0
        if ref is not None:
            ref = require_device_tensor(ref, self.shape, self.tdtype, self.device, "ref").contiguous()
            ref_ptr = ref.data_ptr()
        return qlga_observable_sums(self.handle, y0, self.shape[1] if y1 is None else y1, ref_ptr)

    def fields(self):
        """Per-site fields, numpy (11, ny, nx): F_par, F_perp, |A00|, r, g, b, vorticity m=+2..-2."""
        out = np.empty((11, self.shape[1], self.shape[2]), dtype=self.dtype)
        qlga_fields(self.handle, out.ctypes.data, QLGA_HOST)
        return out

    # -- adjoint (reverse mode)
    def adjoint_workspace(self, nsteps, checkpoint_every=100):
        """Device workspace (torch uint8 tensor) for an adjoint run of nsteps; pass it to
        adjoint_forward / adjoint_backward."""
        nb = qlga_adjoint_workspace_bytes(self.cfg, nsteps, checkpoint_every)
        return self._torch.empty(nb + 256, dtype=self._torch.uint8, device=self.device), nb

    def _device_tensor(self, t):
        return require_device_tensor(t, self.shape, self.tdtype, self.device, "tensor").contiguous()

    def adjoint_forward(self, x0, nsteps, checkpoint_every, ws):
        """Load x0 (device tensor), run nsteps plain steps keeping checkpoints in ws."""
        buf, nb = ws
        x0 = self._device_tensor(x0)
        qlga_adjoint_forward(self.handle, x0.data_ptr(), nsteps, checkpoint_every, self._aligned(buf), nb)

    def adjoint_backward(self, cot, nsteps, checkpoint_every, ws):
        """dL/dx_n (device tensor) -> (dL/dx_0 as a new tensor, dL/dg as numpy[3])."""
        buf, nb = ws
        c = self._device_tensor(cot).clone()
        d = qlga_adjoint_backward(self.handle, nsteps, checkpoint_every, self._aligned(buf), nb, c.data_ptr())
        return c, d

    def adjoint_step(self, x, cot):
        """Pull dL/dx_{k+1} back through one plain step at x (device tensors): returns
        (dL/dx_k, dL/dg)."""
        buf, nb = self.adjoint_workspace(1, 1)
        x = self._device_tensor(x)
        c = self._device_tensor(cot).clone()
        d = qlga_adjoint_step(self.handle, x.data_ptr(), c.data_ptr(), self._aligned(buf), nb)
        return c, d

    def gradient(self, x0, nsteps, cot, checkpoint_every=100):
        """dL/dx_0 and dL/dg for L with dL/dx_n = cot, through nsteps plain steps from x0."""
        ws = self.adjoint_workspace(nsteps, checkpoint_every)
        self.adjoint_forward(x0, nsteps, checkpoint_every, ws)
        return self.adjoint_backward(cot, nsteps, checkpoint_every, ws)

    def set_step2d_mode(self, mode):
        """2D kernel form: QLGA_STEP2D_AUTO (default), QLGA_STEP2D_FUSED or QLGA_STEP2D_TWO_PASS."""
        qlga_set_step2d_mode(self.handle, mode)

    def step2d_kernel(self):
        """The 2D kernel form the next step uses (QLGA_STEP2D_FUSED / _TWO_PASS; 0 in 1D)."""
        return qlga_get_step2d_kernel(self.handle)

    def set_1d_shape(self, threads=0, sites_per_thread=0, steps=0):
        """Force the 1D launch shape (see qlga_set_1d_shape); zeros: time the candidates."""
        _check(load_library().qlga_set_1d_shape(_H(self.handle), int(threads), int(sites_per_thread),
                                                int(steps)), "qlga_set_1d_shape")

    def shape_1d(self):
        """(threads, sites per thread, steps per launch) of the fused 1D steps; zeros before tuning."""
        t, spt, st = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load_library().qlga_get_1d_shape(_H(self.handle), ctypes.byref(t), ctypes.byref(spt),
                                                ctypes.byref(st)), "qlga_get_1d_shape")
        return t.value, spt.value, st.value

    def set_graph_steps(self, steps):
        """Steps per CUDA graph replay (even; 0 turns graphs off)."""
        qlga_set_graph_steps(self.handle, steps)

    def synchronize(self):
        qlga_synchronize(self.handle)

    def launch_count(self) -> int:
        return qlga_launch_count(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            qlga_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------------ autograd

_lattice_cache = {}


def _lattice_for(shape, dtype, g, kinetic_variant, device):
    import torch
    ny, nx = int(shape[1]), int(shape[2])
    key = (ny, nx, dtype, tuple(float(v) for v in g), int(kinetic_variant), str(device))
    lat = _lattice_cache.get(key)
    if lat is None or lat.handle is None:
        if len(_lattice_cache) > 8:
            _lattice_cache.clear()
        lat = Lattice(1 if ny == 1 else 2, nx, ny, 32 if dtype == torch.float32 else 64, g,
                      kinetic_variant=kinetic_variant, device=device)
        _lattice_cache[key] = lat
    return lat


def _make_evolve():
    import torch

    class Evolve(torch.autograd.Function):
        """x_n = (K U)^n x_0 on the GPU, differentiable in x_0 and in the couplings g.

        Forward: qlga_adjoint_forward (checkpoints every C steps, held with the function's
        context).  Backward: qlga_adjoint_backward (segment recompute, pull-back)."""

        @staticmethod
        def forward(ctx, x0, g, nsteps, checkpoint_every, kinetic_variant):
            lat = _lattice_for(x0.shape, x0.dtype, g.detach().cpu().tolist(), kinetic_variant, x0.device)
            ws = lat.adjoint_workspace(nsteps, checkpoint_every)
            lat.adjoint_forward(x0.detach(), nsteps, checkpoint_every, ws)
            xn = lat.device_state()
            ctx.lat, ctx.ws, ctx.nsteps, ctx.C = lat, ws, int(nsteps), int(checkpoint_every)
            ctx.g_dtype, ctx.g_device = g.dtype, g.device
            return xn

        @staticmethod
        def backward(ctx, grad_xn):
            lat = ctx.lat
            # the checkpoints stay with ctx: a graph kept with retain_graph may be pulled back again
            cot, d = lat.adjoint_backward(grad_xn.to(lat.tdtype).contiguous(), ctx.nsteps, ctx.C, ctx.ws)
            dg = torch.tensor(d, dtype=ctx.g_dtype, device=ctx.g_device)
            return cot, dg, None, None, None

    return Evolve


_evolve_fn = None


def evolve(x0, g, nsteps, checkpoint_every=100, kinetic_variant=0):
    """Differentiable run of nsteps plain QLGA steps.

    x0: CUDA tensor (5, ny, nx, 2, 2), float64 or float32 (the run's precision); ny = 1 is 1D.
    g: tensor of the couplings (g0, g1, g2).  Returns x_n; gradients flow to x0 and g through the
    library's adjoint (FP64 or FP32 like x0), with checkpoints every checkpoint_every steps."""
    global _evolve_fn
    if _evolve_fn is None:
        _evolve_fn = _make_evolve()
    return _evolve_fn.apply(x0, g, int(nsteps), int(checkpoint_every), int(kinetic_variant))


_objective_fn = None


def _make_objective():
    import torch

    class Objective(torch.autograd.Function):
        """(P_level, singlet fraction, energy) of a state tensor through qlga_objective; the
        backward pass asks the library for the cotangent of the weighted sum the incoming
        gradient defines, and for the energy's own dependence on the couplings."""

        @staticmethod
        def forward(ctx, x, g, level):
            lat = _lattice_for(x.shape, x.dtype, (0.0, 0.0, 0.0), 0, x.device)
            xc = require_device_tensor(x.detach(), lat.shape, lat.tdtype, lat.device, "x").contiguous()
            vals, _ = qlga_objective(lat.handle, xc.data_ptr(), level, g.detach().cpu().double().numpy())
            ctx.save_for_backward(xc, g)
            ctx.level = int(level)
            return torch.tensor(vals, dtype=torch.float64, device=x.device)

        @staticmethod
        def backward(ctx, grad_vals):
            xc, g = ctx.saved_tensors
            lat = _lattice_for(xc.shape, xc.dtype, (0.0, 0.0, 0.0), 0, xc.device)
            cot = torch.empty_like(xc)
            w = grad_vals.detach().double().cpu().numpy()
            _, dg = qlga_objective(lat.handle, xc.data_ptr(), ctx.level, g.detach().cpu().double().numpy(), w,
                                   cot.data_ptr())
            return cot, torch.tensor(dg, dtype=g.dtype, device=g.device), None

    return Objective


def objectives(x, g=(0.0, 0.0, 0.0), level=2):
    """Tensor (P_level, singlet fraction, energy) of a CUDA state tensor (5, ny, nx, 2, 2)
    (float64 or float32; ny = 1 is 1D), differentiable in x and in the couplings g of the energy
    (a tensor or three floats).  Computed by the library (qlga_objective): FP64 sums; the
    cotangent comes from the library's kernel."""
    import torch
    global _objective_fn
    if _objective_fn is None:
        _objective_fn = _make_objective()
    if not (isinstance(x, torch.Tensor) and x.is_cuda):
        raise TypeError("objectives need a CUDA tensor (the library computes them on the GPU)")
    gt = g if isinstance(g, torch.Tensor) else torch.tensor([float(v) for v in g], dtype=torch.float64,
                                                            device=x.device)
    return _objective_fn.apply(x, gt, int(level))


def population(x, level):
    """Objective: qubit-basis population sum |a_m|^2 + |b_m|^2 of level index `level`
    (0..4 for m = +2..-2) of a CUDA state tensor (5, ny, nx, 2, 2)."""
    return objectives(x, level=level)[0]


def singlet_fraction(x):
    """Objective: sum |psi^T J psi|^2 / sum rho^2 of the boson field psi = a + b of a CUDA state
    tensor (5, ny, nx, 2, 2), J with (J psi)_m = (-1)^m psi_{-m}."""
    return objectives(x)[1]


def energy(x, g):
    """Objective: the energy of the boson field psi = a + b of a CUDA state tensor
    (5, ny, nx, 2, 2), as the library's observables define it: sum over sites of sum_axis sum_m
    |psi_m(j+1) - psi_m(j)|^2 (periodic forward differences) + g0/2 rho^2 + g1/2 |F|^2 +
    g2/10 |psi^T J psi|^2.  g: couplings (g0, g1, g2), floats or a tensor (then differentiable)."""
    return objectives(x, g)[2]


# ------------------------------------------------------------------ batches of 1D lattices

def make_batch_config(lengths, couplings, precision=32, epsilon=0.1, kinetic_variant=0,
                      use_graph=True, heights=None):
    """Returns (config, keepalive arrays) -- the arrays must outlive the create call.
    lengths: nx of each run; heights: ny of each run (None: every run is 1D)."""
    L = np.ascontiguousarray(lengths, dtype=np.int64)
    G = np.ascontiguousarray(couplings, dtype=np.float64).reshape(len(L), 3)
    H = None if heights is None else np.ascontiguousarray(heights, dtype=np.int64)
    cfg = QlgaBatchConfig(int(precision), len(L), L.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(epsilon),
                          int(kinetic_variant), int(bool(use_graph)),
                          None if H is None else H.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return cfg, (L, G, H)


def qlga_batch_state_bytes(cfg) -> int:
    out = ctypes.c_size_t()
    _check(load_library().qlga_batch_state_bytes(ctypes.byref(cfg), ctypes.byref(out)),
           "qlga_batch_state_bytes")
    return out.value


class Batch:
    """Many periodic lattices of uneven size (1D runs, and 2D runs in FP32), advanced together.

    The state is the concatenation of the runs' states in the library layout, as a flat
    float32 / float64 array (see inputs.BatchWorkload); run r holds 20 * nx_r * ny_r reals."""

    def __init__(self, lengths, couplings, precision=32, epsilon=0.1, kinetic_variant=0,
                 use_graph=True, stream=None, heights=None):
        import torch
        self.lengths = np.asarray(lengths, dtype=np.int64)
        self.heights = np.ones_like(self.lengths) if heights is None else np.asarray(heights, dtype=np.int64)
        self.nruns = len(self.lengths)
        self.dtype = np.float32 if precision == 32 else np.float64
        cfg, keep = make_batch_config(lengths, couplings, precision, epsilon, kinetic_variant,
                                      use_graph, heights)
        if stream is None:
            # graph capture needs a stream other than the legacy default stream
            stream = torch.cuda.Stream() if use_graph else torch.cuda.current_stream()
        self.stream = stream
        h = _H()
        _check(load_library().qlga_batch_create(ctypes.byref(cfg), _VP(self.stream.cuda_stream),
                                                ctypes.byref(h)), "qlga_batch_create")
        self.handle = h.value
        self.nreals = int((self.lengths * self.heights).sum()) * 20

    def load_state(self, state):
        a = np.ascontiguousarray(state, dtype=self.dtype).ravel()
        if a.size != self.nreals:
            raise ValueError("batch state must hold %d reals, got %d" % (self.nreals, a.size))
        _check(load_library().qlga_batch_load_state(_H(self.handle), _VP(a.ctypes.data), QLGA_HOST),
               "qlga_batch_load_state")

    def get_state(self):
        out = np.empty(self.nreals, dtype=self.dtype)
        _check(load_library().qlga_batch_get_state(_H(self.handle), _VP(out.ctypes.data), QLGA_HOST),
               "qlga_batch_get_state")
        return out

    def step(self, n=1):
        _check(load_library().qlga_batch_step(_H(self.handle), ctypes.c_int64(int(n))), "qlga_batch_step")

    def observables(self):
        arr = (QlgaObs * self.nruns)()
        _check(load_library().qlga_batch_observables(_H(self.handle), arr), "qlga_batch_observables")
        return [obs_to_dict(o) for o in arr]

    def info(self):
        w, spt, l, g, st = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(load_library().qlga_batch_info(_H(self.handle), ctypes.byref(w), ctypes.byref(spt),
                                              ctypes.byref(l), ctypes.byref(g), ctypes.byref(st)),
               "qlga_batch_info")
        return {"tile_width": w.value, "sites_per_thread": spt.value, "launches": l.value,
                "graph_steps": g.value, "steps_per_launch": st.value}

    def set_shape(self, threads=0, sites_per_thread=0, steps=0):
        """Force the 1D runs' launch shape (see qlga_batch_set_shape); zeros: time the candidates."""
        _check(load_library().qlga_batch_set_shape(_H(self.handle), int(threads), int(sites_per_thread),
                                                   int(steps)), "qlga_batch_set_shape")

    def close(self):
        if getattr(self, "handle", None):
            _check(load_library().qlga_batch_destroy(_H(self.handle)), "qlga_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


Batch1D = Batch  # the 1D-only name
