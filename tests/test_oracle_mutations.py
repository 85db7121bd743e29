"""Plant a plausible mistake in a copy of the oracle source and check that a pin catches it.

Each case edits one line of the oracle (a dropped sign, a flipped exponent, a reversed
stream, a reordered block, a halved term, a conjugation slip), compiles the copy with gcc
and runs the pin that should fail.  The real oracle is never modified.
"""
import pytest

import oracle
import pins

MUTATIONS = [
    # (id, original text, replacement, pin that must fail, its pass threshold)
    ("singlet_sign", "const double sign = (m % 2 == 0) ? 1.0 : -1.0;\n        s[i]",
     "const double sign = 1.0;\n        s[i]", lambda o: pins.pin_table1(o), 1e-13),
    ("spin_term_half", "v += g1 * F[nu] * f[nu][i][j];", "v += 0.5 * g1 * F[nu] * f[nu][i][j];",
     lambda o: pins.pin_table1(o), 1e-13),
    ("exp_sign", "cexp(-I * delta * lam[k])", "cexp(I * delta * lam[k])",
     lambda o: pins.pin_tf_phase(o), 1e-13),
    ("jacobi_conj", "Gqp = -s * conj(u)", "Gqp = -s * u", lambda o: pins.pin_expm(o), 1e-13),
    ("stream_direction", "sx = ((x - dir) % nx + nx) % nx;", "sx = ((x + dir) % nx + nx) % nx;",
     lambda o: pins.pin_plane_wave_symbol(o), 1e-13),
    ("block_order", "block_qubit[4] = {1, 1, 0, 0};", "block_qubit[4] = {0, 0, 1, 1};",
     lambda o: pins.pin_dense_step(o, 1), 1e-13),
    ("collide_transposed", "C[0][0] = 0.5 * (1.0 - I); C[0][1] = 0.5 * (1.0 + I);",
     "C[0][0] = 0.5 * (1.0 + I); C[0][1] = 0.5 * (1.0 - I);",
     lambda o: pins.pin_plane_wave_symbol(o), 1e-13),
    ("potential_uses_a_only", "\n            psi[m] = a[m] + b[m];", "\n            psi[m] = a[m] + a[m];",
     lambda o: pins.pin_dense_step(o, 2), 1e-13),
    ("y_stream_on_x", "else sy = ((y - dir) % ny + ny) % ny;", "else sx = ((x - dir) % nx + nx) % nx;",
     lambda o: pins.pin_plane_wave_symbol(o), 1e-13),
    ("vorticity_sign", "w = (vy_xp - vy_xm - vx_yp + vx_ym) / 2.0;", "w = (vy_xp - vy_xm + vx_yp - vx_ym) / 2.0;",
     lambda o: pins.pin_fields(o), 1e-12),
    ("interleave_fraction", "const double frac = 1.0 / (4.0 * cfg->ndim);",
     "const double frac = 1.0 / 4.0;", lambda o: pins.pin_dense_step(o, 2, interleave=1), 1e-13),
    # adjoint
    ("frechet_phase_sign", "cexp(-I * delta * 0.5 * (li + lj))", "cexp(I * delta * 0.5 * (li + lj))",
     lambda o: pins.pin_frechet(o), 1e-12),
    ("adjoint_stream_direction", "stream(st, cfg, axis, q, -1);     /* (S_c)^dagger",
     "stream(st, cfg, axis, q, +1);     /* (S_c)^dagger", lambda o: pins.pin_kinetic_adjoint(o), 1e-13),
    ("adjoint_collide_not_conjugated", "collide_any(st, cfg, 0, 1);       /* C^dagger */",
     "collide_any(st, cfg, 0, 0);       /* C^dagger */", lambda o: pins.pin_kinetic_adjoint(o), 1e-13),
    ("adjoint_axes_forward_order", "for (int axis = cfg->ndim - 1; axis >= 0; --axis)\n        for (int k = 3;",
     "for (int axis = 0; axis < cfg->ndim; ++axis)\n        for (int k = 3;", lambda o: pins.pin_kinetic_adjoint(o), 1e-13),
    ("adjoint_H_hermitian_part", "H[i][j] = (G[i][j] - conj(G[j][i])) / (2.0 * I);",
     "H[i][j] = (G[i][j] + conj(G[j][i])) / 2.0;", lambda o: pins.pin_vjp_fd(o, "potential"), 1e-8),
    ("adjoint_singlet_dropped", "h += (2.0 * cfg->g2 / 5.0) *", "h += 0.0 * (2.0 * cfg->g2 / 5.0) *",
     lambda o: pins.pin_vjp_fd(o, "potential"), 1e-8),
    ("adjoint_spin_half", "h += 2.0 * cfg->g1 * trfH[nu]", "h += cfg->g1 * trfH[nu]",
     lambda o: pins.pin_vjp_fd(o, "step"), 1e-8),
    ("adjoint_missing_U_dagger", "pa[i] += conj(U[j][i]) * ga[j];", "pa[i] += U[j][i] * ga[j];",
     lambda o: pins.pin_vjp_fd(o, "potential"), 1e-8),
    ("adjoint_psi_uses_a_only", "++m) psi[m] = a[m] + b[m];", "++m) psi[m] = a[m] + a[m];",
     lambda o: pins.pin_vjp_fd(o, "potential"), 1e-8),
    ("coupling_g2_fifth", "dcoup[2] += delta * creal(sHs) / 5.0;", "dcoup[2] += delta * creal(sHs);",
     lambda o: pins.pin_coupling_fd(o), 1e-7),
    # observables and per-site fields
    ("energy_spin_term_full", "0.5 * cfg->g1 * F2", "cfg->g1 * F2", lambda o: pins.pin_observables(o), 1e-12),
    ("energy_singlet_fifth", "0.1 * cfg->g2 * th2", "0.2 * cfg->g2 * th2", lambda o: pins.pin_observables(o), 1e-12),
    ("energy_gradient_x_only", "for (int axis = 0; axis < cfg->ndim; ++axis) {\n                const long xn",
     "for (int axis = 0; axis < 1; ++axis) {\n                const long xn", lambda o: pins.pin_observables(o), 1e-12),
    ("singlet_without_sqrt5", "out[9] += creal(theta) / sqrt(5.0);", "out[9] += creal(theta);",
     lambda o: pins.pin_observables(o), 1e-12),
    ("magnetisation_sign", "out[7] += (2 - m) * pm;", "out[7] += (m - 2) * pm;", lambda o: pins.pin_observables(o), 1e-12),
    ("overlap_unconjugated", "const cplx ov = conj(psi[m]) * r;", "const cplx ov = psi[m] * r;",
     lambda o: pins.pin_observables(o), 1e-12),
    ("a00_without_sqrt5", "const double a00 = cabs(theta) / sqrt(5.0);", "const double a00 = cabs(theta);",
     lambda o: pins.pin_fields(o), 1e-12),
    ("fperp_with_fz", "fperp = sqrt(F[0] * F[0] + F[1] * F[1]);", "fperp = sqrt(F[0] * F[0] + F[2] * F[2]);",
     lambda o: pins.pin_fields(o), 1e-12),
    ("colour_unnormalised", "out[3 * n + site] = nrm > 0 ? fabs(fpar) / nrm : 0.0;",
     "out[3 * n + site] = nrm > 0 ? fabs(fpar) : 0.0;", lambda o: pins.pin_fields(o), 1e-12),
]


@pytest.mark.parametrize("mid,old,new,pin,tol", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(tmp_path, mid, old, new, pin, tol):
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor not found exactly once: %s" % mid
    path = oracle.compile_source(src.replace(old, new), str(tmp_path / ("liboracle_%s.so" % mid)))
    mutant = oracle.Oracle(path)
    assert pin(mutant) > tol, "pin did not catch mutation %s" % mid
