"""The FP64 kernels evaluate the Taylor polynomials of U = exp(-i delta W) (and, in the pull-back,
of its Frechet derivative) with the Horner steps of order above k0 in FP32 and the k0 outer steps
in FP64 on the exact input, k0 >= 1 the smallest order with beta^k0 / k0! <= tau (tau = 2^-31
for U, 2^-38 for the pull-back; beta >= ||delta W||).  This CPU test restates that split in numpy
(complex64 inner steps, complex128 outer steps) and checks the claim it rests on: the result
stays within FP64 rounding of the all-FP64 polynomial, for Hermitian 5x5 matrices of the norms
the lattices produce and for inputs of any scale.  No oracle and no GPU: a check of the error
bound, not of the kernels (the GPU parity tests check those against the oracle).  Measured with
these generators: the worst case is 1.6 x 2^-53 for U at 2^-31; the Frechet series would reach
45 x 2^-53 at 2^-31, and stays at 2.7 x 2^-53 at the 2^-38 the pull-back uses."""
import math

import numpy as np
import pytest

TAU_U = 2.0 ** -31
TAU_ADJ = 2.0 ** -38
TOL64 = 2.0 ** -53


def degree(beta, tol):
    """Smallest K with beta^(K+1)/(K+1)! <= tol (the kernels' taylor_degree)."""
    K, term = 0, beta
    while term > tol and K < 40:
        K += 1
        term *= beta / (K + 1)
    return K


def split(beta, K, tau):
    k0 = degree(beta, tau) + 1
    return min(k0, K)


def horner(A, x, K, k0):
    """sum_{j<=K} A^j x / j! by Horner steps v <- x + A v / k, k = K .. 1; the steps k > k0 in
    complex64 (A and x rounded to it), the rest in complex128 on the exact x."""
    v = x.astype(np.complex64)
    A32, x32 = A.astype(np.complex64), x.astype(np.complex64)
    k = K
    while k > k0:
        v = x32 + (A32 @ v) * np.float32(1.0 / k)
        k -= 1
    v = v.astype(np.complex128)
    while k >= 1:
        v = x + (A @ v) / k
        k -= 1
    return v


def random_w(rng, beta):
    """A Hermitian 5x5 matrix of spectral norm beta."""
    h = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
    h = (h + h.conj().T) / 2
    return beta * h / np.linalg.norm(h, 2)


@pytest.mark.parametrize("beta", [1e-3, 1e-2, 0.05, 0.1, 0.3, 1.0])
def test_inner_fp32_steps_stay_within_fp64_rounding(beta):
    rng = np.random.default_rng(int(beta * 1e6) + 7)
    for trial in range(200):
        W = random_w(rng, beta)
        A = -1j * W
        scale = 10.0 ** rng.uniform(-6, 3)
        x = scale * (rng.normal(size=5) + 1j * rng.normal(size=5))
        K = degree(beta, TOL64)
        k0 = split(beta, K, TAU_U)
        assert 1 <= k0 <= K
        mixed = horner(A, x, K, k0)
        full = horner(A, x, K, K)          # k0 = K: every step in FP64
        err = np.linalg.norm(mixed - full) / np.linalg.norm(x)
        assert err <= 4 * TOL64, (beta, trial, K, k0, err)


def test_split_moves_terms_to_fp32_at_the_lattices_norms():
    """At the norms of the vortex lattices (beta ~ 0.01-0.1) the split leaves some steps in FP32."""
    for beta in (0.01, 0.05, 0.1):
        K = degree(beta, TOL64)
        assert split(beta, K, TAU_U) < K
        assert split(beta, K, TAU_ADJ) <= K


def frechet_augmented(A, E, s, K, k0):
    """The upper block of the Taylor polynomial of [[A, E], [0, A]] on [0; s] (the pull-back's
    augmented Horner), with the split of horner()."""
    M = np.zeros((10, 10), dtype=np.complex128)
    M[:5, :5] = A
    M[:5, 5:] = E
    M[5:, 5:] = A
    z = np.concatenate([np.zeros(5, dtype=np.complex128), s])
    return horner(M, z, K, k0)[:5]


@pytest.mark.parametrize("beta", [1e-2, 0.05, 0.1, 0.3])
def test_inner_fp32_steps_of_the_frechet_series(beta):
    rng = np.random.default_rng(int(beta * 1e6) + 11)
    for trial in range(200):
        A = -1j * random_w(rng, beta)
        # E: the kind of matrix the pull-back uses (a spin matrix times the site, or a rank-two
        # product of the state and its cotangent), of norm up to ~2
        e = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
        E = -1j * 2.0 * e / np.linalg.norm(e, 2)
        s = rng.normal(size=5) + 1j * rng.normal(size=5)
        K = degree(beta, TOL64)
        k0 = split(beta, K, TAU_ADJ)
        mixed = frechet_augmented(A, E, s, K, k0)
        full = frechet_augmented(A, E, s, K, K)
        err = np.linalg.norm(mixed - full) / (np.linalg.norm(s) * math.e ** beta)
        assert err <= 8 * TOL64, (beta, trial, K, k0, err)
