"""Pins of the oracle's adjoint (reverse-mode) functions against what mathematics fixes:
the block-triangular exponential for the Frechet derivative, the adjoint identity of the
unitary kinetic operator, finite differences of the independently pinned forward map, and a
closed-form coupling gradient."""
import pytest

import pins


def test_frechet_exp_matches_block_triangular_exponential():
    assert pins.pin_frechet(pins.oracle.default()) < 1e-12


def test_kinetic_adjoint_identity_and_unitarity():
    assert pins.pin_kinetic_adjoint(pins.oracle.default()) < 1e-13


@pytest.mark.parametrize("what", ["potential", "step", "run"])
def test_vjp_matches_finite_differences(what):
    assert pins.pin_vjp_fd(pins.oracle.default(), what) < 1e-8


def test_coupling_gradient_matches_finite_differences():
    assert pins.pin_coupling_fd(pins.oracle.default()) < 1e-7


def test_coupling_gradient_closed_form_uniform_state():
    assert pins.pin_tf_coupling_gradient(pins.oracle.default()) < 1e-12


def test_interleaved_adjoint_rejected():
    import numpy as np
    cfg = pins.oracle.make_cfg(1, 8, 1, 1.0, 0.1, 0.1, interleave=1)
    x = np.zeros((5, 1, 8, 2, 2))
    with pytest.raises(ValueError):
        pins.oracle.default().vjp_step(x, x.copy(), cfg)
