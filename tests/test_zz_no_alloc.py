"""The allocation-free observables entry point against the allocating one.

Some callers of this library cannot allocate device memory: their memory belongs to their own
allocator or to a fixed memory plan (a cudaMalloc from the library could fail or fragment that
pool), or they run time-critical loops that must not stall on cudaMalloc / cudaFree.  For them
qlga_observables_noalloc() keeps its reduction scratch in a static device array.  This file is
collected last; it calls that entry point through the C ABI, twice in a row on different states,
and checks each result against qlga_observables(): within 1e-12 of the norm for an FP64 state;
within 1e-8 of each quantity's scale for an FP32 state, whose FP32 per-site terms the handle may
form and sum in another order (a 2D state held pending K is read out in one fused pass; the two
differ by ~3e-10) -- far below what a leak of the first call's scratch into the second would leave.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1907_12834_gb300 import inputs as I  # noqa: E402
from paper_1907_12834_gb300 import qlga  # noqa: E402

KEYS = ("norm_qubit", "norm_boson", "magnetisation", "energy", "singlet_re", "singlet_im",
        "singlet_fraction", "overlap_re", "overlap_im")


def call_noalloc(cfg, state_ptr, ref_ptr, stream):
    lib = qlga.load_library()
    out = qlga.QlgaObs()
    status = lib.qlga_observables_noalloc(ctypes.byref(cfg), ctypes.c_void_p(state_ptr),
                                          ctypes.c_void_p(ref_ptr or None),
                                          ctypes.c_void_p(stream or None), ctypes.byref(out))
    return status, qlga.obs_to_dict(out)


def assert_same(got, want, precision):
    tol = 1e-12 if precision == 64 else 1e-8
    scale = want["norm_qubit"]
    for k in KEYS:
        ks = max(scale, 1.0) if precision == 64 else max(scale, abs(want[k]), 1.0)
        assert abs(got[k] - want[k]) <= tol * ks, (k, got[k], want[k])
    np.testing.assert_allclose(got["pop"], want["pop"], rtol=0, atol=tol * scale)


@pytest.mark.parametrize("precision,ndim,nx,ny", [(32, 2, 300, 257), (64, 1, 5000, 1),
                                                  (32, 2, 1024, 1024), (64, 2, 256, 264),
                                                  (32, 1, 5000, 1)])
def test_noalloc_observables_match_twice_in_a_row(precision, ndim, nx, ny):
    rng = np.random.default_rng(nx + ny + precision)
    g = (1.0, 0.8, -0.6)
    lat = qlga.Lattice(ndim, nx, ny, precision=precision, g=g)
    lat.load_state(I.random_state(rng, nx, ny, scale=0.05).astype(lat.dtype))
    lat.step(2)
    stream = lat.stream.cuda_stream

    # first call: with a reference state for the overlap
    s1 = lat.device_state()
    ref = torch.from_numpy(I.random_state(rng, nx, ny, scale=0.05).astype(lat.dtype)).cuda()
    want1 = lat.observables(ref=ref)
    status, got1 = call_noalloc(lat.cfg, s1.data_ptr(), ref.data_ptr(), stream)
    assert status == qlga.QLGA_OK, qlga.qlga_last_error()
    assert_same(got1, want1, precision)

    # second call, on a later state and without a reference: nothing of the first call leaks in
    lat.step(3)
    s2 = lat.device_state()
    want2 = lat.observables()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    status, got2 = call_noalloc(lat.cfg, s2.data_ptr(), 0, stream)
    free_after = torch.cuda.mem_get_info()[0]
    assert status == qlga.QLGA_OK, qlga.qlga_last_error()
    assert_same(got2, want2, precision)
    assert got2["overlap_re"] == 0.0 and got2["overlap_im"] == 0.0
    assert free_after == free_before
    lat.close()


def test_noalloc_rejects_configurations_beyond_the_limits():
    cfg = qlga.make_config(2, 4, 4, precision=32)          # below the minimum lattice size
    dummy = torch.zeros(64, device="cuda")
    status, _ = call_noalloc(cfg, dummy.data_ptr(), 0, 0)
    assert status == qlga.QLGA_ERR_INVALID_ARG
    cfg = qlga.make_config(2, 1 << 20, 1 << 20, precision=32)   # beyond the lattice maximum
    status, _ = call_noalloc(cfg, dummy.data_ptr(), 0, 0)
    assert status == qlga.QLGA_ERR_INVALID_ARG
    assert qlga.qlga_last_error()
