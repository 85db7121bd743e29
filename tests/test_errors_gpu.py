"""Error paths of the C ABI that need a device.

A lattice larger than the GPU's memory must come back from qlga_create as QLGA_ERR_OOM: the
failed cudaMalloc is an ordinary error return (no fault), every buffer allocated before it is
released, and the CUDA context stays usable for the next lattice.
"""
import numpy as np
import pytest

import oracle
from paper_1907_12834_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1907_12834_gb300 import qlga  # noqa: E402

BYTES_PER_SITE_F64 = 160  # 10 complex FP64 amplitudes


def free_device_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("case", ["first_buffer", "second_buffer"])
def test_lattice_larger_than_memory_is_oom(case):
    """qlga_create allocates two state buffers and a work space.  first_buffer: 2^31 FP64 sites
    (344 GB per buffer) cannot be allocated at all; second_buffer: a buffer of 0.7 of the free
    memory fits once but not twice, so the second allocation fails after the first succeeded and
    the first must be released."""
    torch.cuda.empty_cache()
    free0 = free_device_bytes()
    nx = 1 << 31 if case == "first_buffer" else int(0.7 * free0 / BYTES_PER_SITE_F64)
    cfg = qlga.make_config(1, nx, 1, precision=64)
    assert qlga.qlga_state_bytes(cfg) == BYTES_PER_SITE_F64 * nx
    with pytest.raises(qlga.QlgaError) as ei:
        qlga.qlga_create(cfg)
    assert ei.value.status == qlga.QLGA_ERR_OOM
    assert abs(free_device_bytes() - free0) < (64 << 20)

    # the context is still usable: a small lattice steps and matches the oracle
    g = (1.0, 0.8, -0.6)
    st = I.random_state(np.random.default_rng(5), 64, 1, scale=0.05)
    lat = qlga.Lattice(1, 64, 1, precision=64, g=g)
    lat.load_state(st)
    lat.step(3)
    got = lat.get_state()
    lat.close()
    ref = oracle.step(np.array(st, dtype=np.float64), oracle.make_cfg(1, 64, 1, *g), 3)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12
