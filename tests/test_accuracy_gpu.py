"""Accuracy record of every timed path against the FP64 oracle, at the paths' own precision.

The oracle's results are stored under tests/golden/ by scripts that call only the oracle
(make_path_accuracy.py, make_long_horizon.py); the GPU runs are the benchmark's own accuracy
legs (bench.path_accuracy, bench.long_horizon_record), so the numbers the benchmark line reports
are the ones checked here.

Long runs (config 1 at its full 16384 sites and 20000 steps under both coupling sets, the config 2
recipe on 512^2 for 5000 steps): every checkpoint's relative L2 error against the oracle is held
to the larger of the precision's target (1e-11 FP64, 1e-4 FP32) and what the dynamics does to
rounding-sized differences -- the oracle's own run from a 1e-13 perturbed start grows by a factor
amp(t) by step t, so a per-step rounding difference u injected at every one of t steps can reach
about u t amp(t): u = 1e-15 in FP64 (the oracle's own step is unitary to about 5e-16 per step,
its U coming from a Jacobi eigendecomposition), 1e-7 in FP32.  The numbers are printed (pytest -s) as the record."""
import json
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1907_12834_gb300 import inputs, qlga  # noqa: E402

GOLD = os.path.join(ROOT, "tests", "golden")


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLD, "path_accuracy.npz")), reason="no stored oracle runs")
def test_each_path_against_the_oracle():
    acc = bench.path_accuracy(torch, qlga, inputs)
    print(json.dumps(acc, indent=1))
    assert acc["config0_fp64_1d"]["rel_l2_vs_oracle"] <= 1e-11
    assert acc["config0_fp64_1d"]["norm_drift"] <= 1e-12
    assert acc["interleaved_fp32_2d"]["rel_l2_vs_oracle"] <= 1e-4
    assert acc["batched_fp32_1d"]["rel_l2_vs_oracle"] <= 1e-4
    assert acc["batched_fp32_2d"]["rel_l2_vs_oracle"] <= 1e-4
    assert acc["adjoint_fp64_2d"]["rel_l2_vs_oracle"] <= 1e-10
    assert acc["adjoint_fp64_2d"]["coupling_gradient_rel_vs_oracle"] <= 1e-9
    assert acc["adjoint_fp32_2d"]["rel_l2_vs_oracle"] <= 1e-3
    for k in ("interleaved_fp32_2d", "batched_fp32_1d", "batched_fp32_2d"):
        assert acc[k]["norm_drift"] <= 1e-5, k


@pytest.mark.parametrize("name", inputs.LONG_HORIZON)
def test_long_horizon_record(name):
    if not os.path.exists(os.path.join(GOLD, "long_horizon_%s.npz" % name)):
        pytest.skip("no stored oracle trajectory")
    rec = bench.long_horizon_record(torch, qlga, inputs, names=[name])[name]
    print(json.dumps(rec))
    steps = np.asarray(rec["steps"], dtype=np.float64)
    growth = np.asarray(rec["oracle_perturbed_1e-13"])
    amp = np.maximum.accumulate(growth / inputs.PERTURBATION)
    for prec, u, target in ((64, 1e-15, 1e-11), (32, 1e-7, 1e-4)):
        err = np.asarray(rec["gpu_fp%d_vs_oracle" % prec])
        bound = np.maximum(target, u * np.maximum(steps, 1) * amp)
        assert np.all(err <= bound), (prec, err.tolist(), bound.tolist())
    # the GPU FP64 run amplifies a 1e-13 start no more than the oracle does: the oracle's
    # difference carries its own (larger) rounding, amplified alike, on top of the perturbation
    g_gpu = np.asarray(rec["gpu_fp64_perturbed_1e-13"])
    assert np.all(g_gpu <= 2 * growth + 1e-13), (g_gpu.tolist(), growth.tolist())
    assert rec["gpu_fp64_norm_drift"] <= 2e-15 * steps[-1] + 1e-15     # unitary to FP64 rounding
