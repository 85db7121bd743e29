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
