"""The 2D per-site fields take the vorticity of each level as pi/2 times an integer: with the
phases S0..S3 at the four diagonal neighbours (x+1,y+1), (x+1,y-1), (x-1,y+1), (x-1,y-1), the
central differences of the wrapped phase velocity cancel but for their wraps, so
    w = (wrap(S0-S1) - wrap(S2-S3) - wrap(S0-S2) + wrap(S1-S3)) / 4 = (pi/2) (n01 - n23 - n02 + n13)
with n the wrap count of each difference.  The kernel takes the phases with the FP32 atan2 of the
exact psi and rechecks a site in FP64 when one of its differences lies within 1e-4 of +-pi.

This CPU test restates both in numpy and checks (1) the identity against the FP64 formula the
oracle evaluates, and (2) that the FP32 phases with the recheck give the FP64 counts, on random
amplitudes and on amplitudes placed right at the wrap boundary.  No GPU, no oracle."""
import numpy as np

PI = np.pi


def wrap(d):
    return np.where(d > PI, d - 2 * PI, np.where(d <= -PI, d + 2 * PI, d))


def count(d, pi):
    return np.where(d > pi, -1, np.where(d <= -pi, 1, 0))


def fp64_formula(S):
    S0, S1, S2, S3 = S
    return (wrap(S0 - S1) * 0.5 - wrap(S2 - S3) * 0.5 - wrap(S0 - S2) * 0.5 + wrap(S1 - S3) * 0.5) * 0.5


def kernel_counts(z):
    """z: complex128 (4, n) amplitudes of the four neighbours -> the kernel's integer N."""
    pf = np.float32(np.pi)
    S = np.arctan2(z.imag.astype(np.float32), z.real.astype(np.float32))
    d = [S[0] - S[1], S[2] - S[3], S[0] - S[2], S[1] - S[3]]
    N = count(d[0], pf) - count(d[1], pf) - count(d[2], pf) + count(d[3], pf)
    near = np.zeros(z.shape[1], dtype=bool)
    for di in d:
        near |= np.abs(np.abs(di) - pf) < np.float32(1e-4)
    S64 = np.arctan2(z.imag, z.real)
    N64 = (count(S64[0] - S64[1], PI) - count(S64[2] - S64[3], PI) - count(S64[0] - S64[2], PI)
           + count(S64[1] - S64[3], PI))
    return np.where(near, N64, N), N64


def test_vorticity_is_pi_over_two_times_the_wrap_counts():
    rng = np.random.default_rng(3)
    S = rng.uniform(-PI, PI, size=(4, 100000))
    S0, S1, S2, S3 = S
    N = count(S0 - S1, PI) - count(S2 - S3, PI) - count(S0 - S2, PI) + count(S1 - S3, PI)
    np.testing.assert_allclose(fp64_formula(S), (PI / 2) * N, rtol=0, atol=4e-15)
    assert set(np.unique(N)) <= {-2, -1, 0, 1, 2}


def test_fp32_phases_with_the_recheck_give_the_fp64_counts():
    rng = np.random.default_rng(5)
    n = 200000
    mag = 10.0 ** rng.uniform(-12, 2, size=(4, n))
    z = mag * np.exp(1j * rng.uniform(-PI, PI, size=(4, n)))
    N, N64 = kernel_counts(z)
    np.testing.assert_array_equal(N, N64)
    # pairs placed right at the wrap boundary: S0 - S1 = +-pi to within a few 1e-9 rad
    base = rng.uniform(-PI, PI, size=n)
    eps = rng.uniform(-5e-9, 5e-9, size=n)
    z = np.stack([np.exp(1j * base), np.exp(1j * (base - PI + eps)),
                  np.exp(1j * rng.uniform(-PI, PI, size=n)), np.exp(1j * rng.uniform(-PI, PI, size=n))])
    N, N64 = kernel_counts(z)
    np.testing.assert_array_equal(N, N64)
