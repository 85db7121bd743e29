"""How far the FP64 oracle's own rounding carries it, measured against the same source evaluated
in long double (oracle.step_long_double: every `double` of the C source made `long double`).

Both builds run the same algorithm on the same discrete operator, so this pins no physics; it
bounds the oracle's accuracy as a reference.  The bound matters when GPU-oracle differences are
read: over a two-soliton run the FP64 oracle drifts from the extended-precision evaluation by
about 7e-16 per step (its U is a sum of eigenprojectors weighted by e^{-i lambda_k}), which sets
the floor below which a GPU-oracle difference says nothing about the GPU.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1907_12834_gb300 import inputs as I


def test_fp64_oracle_against_long_double_build():
    if ctypes.sizeof(ctypes.c_longdouble) <= 8:
        pytest.skip("long double is no wider than double on this platform")
    g = (1.0, 0.8, -0.6)
    w = I.config1(L=1024, couplings=g)
    cfg = oracle.make_cfg(1, w.nx, 1, *g)
    x0 = np.ascontiguousarray(w.state, dtype=np.float64)
    assert np.array_equal(oracle.step_long_double(x0, cfg, 0), x0)  # conversions are exact
    ref = oracle.step_long_double(x0, cfg, 200)
    got = oracle.step(x0.copy(), cfg, 200)
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert 0.0 < rel <= 5e-13, rel  # measured 1.4e-13; nonzero: the long-double build is wider
