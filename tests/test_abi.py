"""The C-ABI library builds, loads and exports every entry point of include/qlga.h; its host-side
argument checking works without a GPU (no compute calls here)."""
import ctypes
import subprocess

import pytest

from paper_1907_12834_gb300 import build as qbuild
from paper_1907_12834_gb300 import qlga


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return qlga.load_library()


def test_exports_every_header_symbol(lib):
    names = qlga.header_symbols()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", qlga.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_state_and_workspace_bytes(lib):
    cfg = qlga.make_config(2, 4096, 4096, precision=32)
    assert qlga.qlga_state_bytes(cfg) == 4096 * 4096 * 20 * 4
    assert qlga.qlga_workspace_bytes(cfg) >= qlga.qlga_state_bytes(cfg)
    cfg = qlga.make_config(1, 1024, 1, precision=64)
    assert qlga.qlga_state_bytes(cfg) == 1024 * 20 * 8


@pytest.mark.parametrize("kw", [
    dict(ndim=3, nx=16, ny=16), dict(ndim=1, nx=4, ny=1), dict(ndim=1, nx=64, ny=2),
    dict(ndim=2, nx=64, ny=4), dict(ndim=2, nx=64, ny=64, precision=16),
    dict(ndim=1, nx=64, ny=1, interleave=2), dict(ndim=1, nx=64, ny=1, kinetic_variant=5),
    dict(ndim=1, nx=64, ny=1, g=(float("nan"), 0, 0)),
])
def test_invalid_configs_rejected(lib, kw):
    with pytest.raises(qlga.QlgaError) as ei:
        qlga.qlga_state_bytes(qlga.make_config(**kw))
    assert ei.value.status == qlga.QLGA_ERR_INVALID_ARG
    assert qlga.qlga_last_error()


def test_null_arguments_rejected(lib):
    assert lib.qlga_step(None, 1) == qlga.QLGA_ERR_INVALID_ARG
    assert lib.qlga_observables(None, None, None) == qlga.QLGA_ERR_INVALID_ARG
    assert lib.qlga_load_state(None, None, 0) == qlga.QLGA_ERR_INVALID_ARG
    assert lib.qlga_destroy(None) == qlga.QLGA_OK
    cfg = qlga.make_config(1, 64)
    assert lib.qlga_state_bytes(ctypes.byref(cfg), None) == qlga.QLGA_ERR_INVALID_ARG


def test_status_strings(lib):
    for s in range(7):
        assert qlga.qlga_status_string(s)
    assert qlga.qlga_status_string(99) == "unknown status"


@pytest.mark.parametrize("kw,status", [
    (dict(lengths=[]), qlga.QLGA_ERR_INVALID_ARG),                              # empty batch
    (dict(lengths=[64, 7]), qlga.QLGA_ERR_INVALID_ARG),                         # run below 8 sites
    (dict(lengths=[(1 << 30) + 1]), qlga.QLGA_ERR_INVALID_ARG),                 # 1D run above 2^30
    (dict(lengths=[1 << 30] * 17), qlga.QLGA_ERR_INVALID_ARG),                  # batch above 2^34 sites
    (dict(lengths=[40], heights=[16]), qlga.QLGA_ERR_INVALID_ARG),              # 2D nx not a multiple of 32
    (dict(lengths=[64], heights=[4]), qlga.QLGA_ERR_INVALID_ARG),               # 2D ny below 8
    (dict(lengths=[64], heights=[16], precision=64), qlga.QLGA_ERR_UNSUPPORTED),  # 2D runs are FP32 only
    (dict(lengths=[64], g=[(float("nan"), 0.0, 0.0)]), qlga.QLGA_ERR_INVALID_ARG),
    (dict(lengths=[64], kinetic_variant=5), qlga.QLGA_ERR_INVALID_ARG),
    (dict(lengths=[64], precision=16), qlga.QLGA_ERR_INVALID_ARG),
])
def test_invalid_batches_rejected_before_any_device_call(lib, kw, status):
    kw = dict(kw)
    lengths = kw.pop("lengths")
    g = kw.pop("g", [(1.0, 0.1, 0.2)] * len(lengths))
    cfg, keep = qlga.make_batch_config(lengths, g, **kw)
    with pytest.raises(qlga.QlgaError) as ei:
        qlga.qlga_batch_state_bytes(cfg)
    assert ei.value.status == status
    h = ctypes.c_void_p()
    assert lib.qlga_batch_create(ctypes.byref(cfg), None, ctypes.byref(h)) == status
    assert not h.value
    del keep


def test_batch_state_bytes(lib):
    cfg, keep = qlga.make_batch_config([64, 100, 64], [(1.0, 0.1, 0.2)] * 3, heights=[1, 1, 16])
    assert qlga.qlga_batch_state_bytes(cfg) == 80 * (64 + 100 + 64 * 16)
    cfg, keep = qlga.make_batch_config([8, 4096], [(1.0, 0.1, 0.2)] * 2, precision=64)
    assert qlga.qlga_batch_state_bytes(cfg) == 160 * (8 + 4096)


def test_create_rejects_bad_arguments_before_allocating(lib):
    h = ctypes.c_void_p()
    bad = qlga.make_config(1, 4)
    assert lib.qlga_create(ctypes.byref(bad), None, ctypes.byref(h)) == qlga.QLGA_ERR_INVALID_ARG
    assert not h.value
    good = qlga.make_config(1, 64)
    assert lib.qlga_create(ctypes.byref(good), None, None) == qlga.QLGA_ERR_INVALID_ARG


def test_adjoint_workspace_bytes(lib):
    """Work space of a checkpointed adjoint run: four state-sized buffers, one checkpoint per
    C steps and a segment of up to C recomputed states, plus a fixed block of partial sums."""
    cfg = qlga.make_config(2, 512, 512, precision=32)
    state = qlga.qlga_state_bytes(cfg)      # a multiple of 256: no alignment padding between states
    fixed = set()
    for n, c in ((200, 100), (200, 50), (200, 200), (200, 1), (1, 1), (0, 5), (25, 7)):
        nck = -(-n // c) if n > 0 else 0
        slots = min(c, n) if n > 0 else 1
        fixed.add(qlga.qlga_adjoint_workspace_bytes(cfg, n, c) - state * (4 + nck + slots))
    assert len(fixed) == 1 and 0 < fixed.pop() < (1 << 20)
    for nsteps, every in ((-1, 10), (10, 0)):
        with pytest.raises(qlga.QlgaError) as ei:
            qlga.qlga_adjoint_workspace_bytes(cfg, nsteps, every)
        assert ei.value.status == qlga.QLGA_ERR_INVALID_ARG


def test_buffer_checks_of_the_binding():
    """The binding refuses buffers the library would read or write past: wrong dtype, shape,
    layout, a read-only output, or a host tensor where a device tensor is required."""
    import numpy as np
    torch = pytest.importorskip("torch")
    shape = (5, 3, 8, 2, 2)
    ok = np.zeros(shape, np.float32)
    assert qlga.require_host_array(ok, shape, np.float32, "x", writable=True) is ok
    bad = [np.zeros(shape, np.float64), np.zeros((5, 3, 9, 2, 2), np.float32),
           np.zeros((5, 8, 3, 2, 2), np.float32).transpose(0, 2, 1, 3, 4)]
    for a in bad:
        with pytest.raises(ValueError):
            qlga.require_host_array(a, shape, np.float32, "x")
    ro = np.zeros(shape, np.float32)
    ro.setflags(write=False)
    qlga.require_host_array(ro, shape, np.float32, "x")
    with pytest.raises(ValueError):
        qlga.require_host_array(ro, shape, np.float32, "x", writable=True)
    with pytest.raises(TypeError):
        qlga.require_device_tensor(torch.zeros(shape), shape, torch.float32, torch.device("cuda", 0), "x")


def test_obs_from_sums_forms_the_observables(lib):
    """qlga_obs_from_sums (host only) against the oracle's observables of a random 2D state: the 14
    sums in the ABI's order go in, the magnetisation sum_m m pop[m] and the singlet fraction
    sum |psi^T J psi|^2 / sum rho^2 come out as the oracle forms them (Sec. III.B Eq. cmap)."""
    import numpy as np
    import oracle
    from paper_1907_12834_gb300 import inputs

    rng = np.random.default_rng(77)
    nx, ny = 12, 9
    st = np.ascontiguousarray(inputs.random_state(rng, nx, ny, scale=0.2), dtype=np.float64)
    ref = np.ascontiguousarray(inputs.random_state(rng, nx, ny, scale=0.2), dtype=np.float64)
    o = oracle.observables(st, oracle.make_cfg(2, nx, ny, 1.0, 0.8, -0.6), ref=ref)
    sums = np.array([o["norm_qubit"], o["norm_boson"], *o["pop"], o["energy"], o["singlet_re"],
                     o["singlet_im"], o["theta2_sum"], o["rho2_sum"], o["overlap_re"], o["overlap_im"]])
    d = qlga.obs_to_dict(qlga.qlga_obs_from_sums(sums, 17))
    assert d["step"] == 17
    assert abs(d["magnetisation"] - o["magnetisation"]) <= 1e-13 * o["norm_qubit"]
    assert d["singlet_fraction"] == pytest.approx(o["singlet_fraction"], rel=1e-15)
    for k in ("norm_qubit", "norm_boson", "energy", "singlet_re", "singlet_im", "overlap_re", "overlap_im"):
        assert d[k] == o[k]
    np.testing.assert_array_equal(d["pop"], o["pop"])
    # an all-zero field has no singlet fraction to form: 0, not a division by zero
    assert qlga.obs_to_dict(qlga.qlga_obs_from_sums(np.zeros(14)))["singlet_fraction"] == 0.0
    bad = sums.copy()
    bad[7] = float("nan")                     # the energy
    with pytest.raises(qlga.QlgaError) as ei:
        qlga.qlga_obs_from_sums(bad)
    assert ei.value.status == qlga.QLGA_ERR_NOT_FINITE
    assert lib.qlga_obs_from_sums(None, 0, None) == qlga.QLGA_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        qlga.qlga_obs_from_sums(sums[:13])
