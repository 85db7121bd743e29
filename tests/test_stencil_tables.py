"""The kinetic stencil tables the kernels are compiled with, checked on the CPU against the
oracle's operators (Sec. VII.B: one axis is the four blocks I'_1 I'_1 I'_2 I'_2 with
I'_c = S_c C' S^T_c C, the I'_2 blocks first; in 2D x then y).

`tests/stencil_tables.cu` is built with nvcc for the host and prints the compile-time tables:
the forward nine-point stencil in the (a, bt = i b) basis, its form on a state held as
(P, Q) = (a + bt, a - bt), and the adjoint stencil of the pull-back.  This test applies each
table to random states with numpy, with the convention the kernels use
(out_dst(j) = 1/16 sum_k g[dst][src][k + 4] in_src(j + k)), and compares with the oracle's
kinetic operator and its adjoint on ragged 1D rings and 2D tori, for both collide readings.  It
also checks the counts of nonzero taps per level (32 in (a, bt), 24 in (P, Q)) and that no
invertible 2 x 2 integer basis with entries in -2..2 gives fewer.  No GPU is used."""
import itertools
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1907_12834_gb300 import build as qbuild

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("stencil") / "stencil_tables")
    cmd = [qbuild._nvcc(), "-std=c++17", "--expt-relaxed-constexpr",
           "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", qbuild.CSRC, "-I", os.path.join(ROOT, "include"),
           "-o", exe, os.path.join(HERE, "stencil_tables.cu")]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("nvcc not found")
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    t = json.loads(out)
    return {k: np.array(v, dtype=np.int64) for k, v in t.items()}   # [variant][dst][src][k]


def random_state(rng, nx, ny):
    return np.ascontiguousarray(rng.standard_normal((5, ny, nx, 2, 2)))


def split(st):
    z = st[..., 0] + 1j * st[..., 1]          # (5, ny, nx, 2): the pair (a, b)
    return z[..., 0], 1j * z[..., 1]          # a, bt = i b


def join(a, bt):
    b = -1j * bt
    out = np.empty(a.shape + (2, 2))
    out[..., 0, 0], out[..., 0, 1] = a.real, a.imag
    out[..., 1, 0], out[..., 1, 1] = b.real, b.imag
    return out


def apply_table(g, u, v, axis):
    """One axis: out_dst(j) = 1/16 sum_k (g[dst][0][k] u(j + k - 4) + g[dst][1][k] v(j + k - 4))."""
    o0 = np.zeros_like(u)
    o1 = np.zeros_like(u)
    for k in range(9):
        su = np.roll(u, -(k - 4), axis=axis)
        sv = np.roll(v, -(k - 4), axis=axis)
        o0 += g[0][0][k] * su + g[0][1][k] * sv
        o1 += g[1][0][k] * su + g[1][1][k] * sv
    return o0 / 16, o1 / 16


AXIS_X, AXIS_Y = 2, 1      # of the (5, ny, nx) complex planes
SHAPES = [(1, 13, 1), (1, 9, 1), (1, 40, 1), (2, 11, 9), (2, 16, 10)]


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("ndim,nx,ny", SHAPES)
def test_forward_table_is_the_oracle_kinetic_operator(tables, variant, ndim, nx, ny):
    rng = np.random.default_rng(100 * nx + ny + variant)
    st = random_state(rng, nx, ny)
    a, bt = split(st)
    g = tables["forward"][variant]
    a, bt = apply_table(g, a, bt, AXIS_X)
    if ndim == 2:
        a, bt = apply_table(g, a, bt, AXIS_Y)
    ref = st.copy()
    oracle.apply_kinetic(ref, oracle.make_cfg(ndim, nx, ny, 1.0, 0.0, 0.0, kinetic_variant=variant))
    np.testing.assert_allclose(join(a, bt), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("ndim,nx,ny", SHAPES)
def test_pq_table_on_the_held_form(tables, variant, ndim, nx, ny):
    """The x axis of the fused kernels reads the held pair (P, Q) = (a + bt, a - bt) with the (P, Q)
    table and writes (a, bt); the y axis then runs on (a, bt) as before."""
    rng = np.random.default_rng(7 * nx + ny + variant)
    st = random_state(rng, nx, ny)
    a, bt = split(st)
    a, bt = apply_table(tables["forward_pq"][variant], a + bt, a - bt, AXIS_X)
    if ndim == 2:
        a, bt = apply_table(tables["forward"][variant], a, bt, AXIS_Y)
    ref = st.copy()
    oracle.apply_kinetic(ref, oracle.make_cfg(ndim, nx, ny, 1.0, 0.0, 0.0, kinetic_variant=variant))
    np.testing.assert_allclose(join(a, bt), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("ndim,nx,ny", SHAPES)
def test_adjoint_table_is_the_oracle_adjoint(tables, variant, ndim, nx, ny):
    """K^dagger: the axes in reverse order (y first in 2D), each by the adjoint table."""
    rng = np.random.default_rng(11 * nx + ny + variant)
    st = random_state(rng, nx, ny)
    a, bt = split(st)
    g = tables["adjoint"][variant]
    if ndim == 2:
        a, bt = apply_table(g, a, bt, AXIS_Y)
    a, bt = apply_table(g, a, bt, AXIS_X)
    ref = st.copy()
    oracle.vjp_kinetic(ref, oracle.make_cfg(ndim, nx, ny, 1.0, 0.0, 0.0, kinetic_variant=variant))
    np.testing.assert_allclose(join(a, bt), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("variant", [0, 1])
def test_adjoint_table_is_the_transpose_of_the_forward_table(tables, variant):
    """The coefficients are real, so the adjoint's tap k is the forward tap -k transposed."""
    f, adj = tables["forward"][variant], tables["adjoint"][variant]
    for k in range(9):
        np.testing.assert_array_equal(adj[:, :, k], f[:, :, 8 - k].T)


def nonzero_taps(g, basis):
    """Nonzero 2 x 2 entries of the taps g_k B^-1 summed over k, for a state held as B (a, bt);
    B^-1 = adj(B) / det(B), so the pattern is that of g_k adj(B) (integers, exact)."""
    adj = np.array([[basis[1][1], -basis[0][1]], [-basis[1][0], basis[0][0]]], dtype=np.int64)
    return int(sum(np.count_nonzero(g[:, :, k] @ adj) for k in range(9)))


@pytest.mark.parametrize("variant", [0, 1])
def test_tap_counts_and_the_held_basis(tables, variant):
    g = tables["forward"][variant]
    assert int(np.count_nonzero(g)) == 32
    assert int(np.count_nonzero(tables["forward_pq"][variant])) == 24
    pq = ((1, 1), (1, -1))
    assert nonzero_taps(g, pq) == 24
    best = min(nonzero_taps(g, B) for B in (((p, q), (r, s))
                                            for p, q, r, s in itertools.product(range(-2, 3), repeat=4))
               if B[0][0] * B[1][1] - B[0][1] * B[1][0] != 0)
    assert best == 24
    # the (P, Q) taps are the (a, bt) taps times [[1, 1], [1, -1]] / 2, exactly
    for k in range(9):
        np.testing.assert_array_equal(2 * tables["forward_pq"][variant][:, :, k],
                                      g[:, :, k] @ np.array([[1, 1], [1, -1]]))
