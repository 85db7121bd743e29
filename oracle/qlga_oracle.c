/*
 * qlga_oracle.c -- plain, slow FP64 CPU reference ("oracle") of the spin-2 BEC quantum
 * lattice gas algorithm of Taylor, Smith & Yepez, arXiv:1907.12834.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library calls this file.  It is used by the
 * tests, by the smoke check and by the CPU-baseline leg of the benchmark, and it shares no
 * code, header or constant with the CUDA path.  Every step is written the plain way the
 * paper states it: whole-lattice sweeps, one operator at a time, FP64 complex arithmetic,
 * and the self-interaction unitary taken from a Hermitian eigendecomposition.
 *
 * State layout (same as the library's data format): 5 planes m = +2..-2, each ny*nx sites
 * with x fastest, each site (a.re, a.im, b.re, b.im): element (m, site, q, c) at
 * ((m*nsites + site)*2 + q)*2 + c.  a = qubit 1 of the pair, b = qubit 2 (Sec. III.B, Eq.
 * full_state: two qubits per m_f level).
 *
 * Readings of passages the paper leaves open (the same ones the library documents):
 *  - boson field of level m: psi_m = a_m + b_m;
 *  - potential V(psi) = g0 rho 1 + g1 sum_nu F_nu f_nu + (g2/5) s s^dagger with
 *    F_nu = psi^dagger f_nu psi and s_m = (-1)^m conj(psi_{-m}); this is the right-hand
 *    side of Eq. eomspin2 / eom_component_form written as V(psi) psi, with the singlet
 *    factor of Eq. spinsinglet read as psi^T J psi / 5 (the printed |A00|^2 and the dropped
 *    (-1)^m are typesetting slips: every row of Table I is an eigenvector of this V);
 *  - U = exp(-i delta V(psi)) with V frozen at the current psi, applied to a and to b;
 *  - collide K1: C = 1/2 [[1-i, 1+i], [1+i, 1-i]], block I'_c = S_c C S^T_c C;
 *    collide K2: C = 1/2 [[1+i, 1-i], [1-i, 1+i]], block I'_c = S_c C^dagger S^T_c C;
 *  - S_c moves qubit c one site toward +x: c(j) <- c(j-1); S^T_c the other way;
 *  - one axis of the kinetic operator is I'_1 I'_1 I'_2 I'_2 (Sec. VII.B), so the I'_2
 *    blocks act first; in 2D the x axis acts before the y axis.
 *
 * Besides the forward step, the file holds the reverse-mode adjoint of the plain step (pull-back
 * of a cotangent through K and through the linearised potential unitary, with the Frechet
 * derivative of the matrix exponential taken in the eigenbasis of V), and per-site diagnostic
 * fields.  Each function states the passage or the derivation it follows.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double kPi = 3.14159265358979323846;

typedef struct oracle_cfg {
    int ndim;              /* 1 or 2 */
    long nx, ny;           /* ny == 1 in 1D */
    double g0, g1, g2;     /* couplings of Eq. hamspin2 */
    int interleave;        /* 0 plain step, 1 interleaved step (Sec. VII.B) */
    int kinetic_variant;   /* 0 = K1, 1 = K2 */
} oracle_cfg;

/* ---------------------------------------------------------------- element access */

static inline double* amp(double* s, long nsites, int m, long site, int q) {
    return s + ((m * nsites + site) * 2 + q) * 2;
}
static inline cplx getc(const double* p) { return p[0] + I * p[1]; }
static inline void putc_(double* p, cplx z) { p[0] = creal(z); p[1] = cimag(z); }

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ---------------------------------------------------------------- spin-2 matrices */

/* f_x, f_y, f_z of Sec. II (the spin-2 SU(2) representation, hbar = 1), rows/columns
 * ordered m = +2..-2. */
static void spin2_matrices(cplx fx[5][5], cplx fy[5][5], cplx fz[5][5]) {
    const double r = sqrt(1.5);
    memset(fx, 0, sizeof(cplx) * 25);
    memset(fy, 0, sizeof(cplx) * 25);
    memset(fz, 0, sizeof(cplx) * 25);
    const double off[4] = {1.0, r, r, 1.0};
    for (int i = 0; i < 4; ++i) {
        fx[i][i + 1] = off[i];
        fx[i + 1][i] = off[i];
        fy[i][i + 1] = -I * off[i];
        fy[i + 1][i] = I * off[i];
    }
    for (int i = 0; i < 5; ++i) fz[i][i] = 2.0 - i;
}

/* V(psi) of Eq. eomspin2 (see the readings above). */
static void potential_matrix(const cplx psi[5], double g0, double g1, double g2, cplx V[5][5]) {
    cplx fx[5][5], fy[5][5], fz[5][5];
    spin2_matrices(fx, fy, fz);
    double rho = 0.0;
    for (int i = 0; i < 5; ++i) rho += creal(conj(psi[i]) * psi[i]);
    double F[3] = {0.0, 0.0, 0.0};
    cplx (*f[3])[5] = {fx, fy, fz};
    for (int nu = 0; nu < 3; ++nu) {
        cplx acc = 0.0;
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) acc += conj(psi[i]) * f[nu][i][j] * psi[j];
        F[nu] = creal(acc);
    }
    cplx s[5];
    for (int i = 0; i < 5; ++i) {
        const int m = 2 - i;
        const double sign = (m % 2 == 0) ? 1.0 : -1.0;
        s[i] = sign * conj(psi[4 - i]); /* psi_{-m} sits at position 4 - i */
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            cplx v = (i == j) ? g0 * rho : 0.0;
            for (int nu = 0; nu < 3; ++nu) v += g1 * F[nu] * f[nu][i][j];
            v += (g2 / 5.0) * s[i] * conj(s[j]);
            V[i][j] = v;
        }
}

/* ------------------------------------------------ Hermitian eigendecomposition (Jacobi)
 *
 * Cyclic Jacobi method for a complex Hermitian matrix.  Each rotation zeroes A[p][q]:
 * with A[p][q] = r e^{i phi}, D = diag(1, e^{-i phi}) on (p, q) makes the pair real, and
 * the real rotation R = [[c, s], [-s, c]] with t = tan(theta) the smaller root of
 * t^2 + 2 tau t - 1 = 0, tau = (A[q][q] - A[p][p]) / (2 r), diagonalises it.  G = D R,
 * A <- G^H A G, Q <- Q G.  On exit A is diagonal (eigenvalues) and the columns of Q are
 * orthonormal eigenvectors.
 */
static void herm_eig(cplx A[5][5], double lam[5], cplx Q[5][5]) {
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Q[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                const double a2 = creal(A[i][j] * conj(A[i][j]));
                tot += a2;
                if (i != j) off += a2;
            }
        if (off == 0.0 || off <= 1e-36 * tot) break;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 5; ++q) {
                const double r = cabs(A[p][q]);
                if (r == 0.0) continue;
                const cplx u = A[p][q] / r;
                const double tau = (creal(A[q][q]) - creal(A[p][p])) / (2.0 * r);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                const cplx Gpp = c, Gpq = s, Gqp = -s * conj(u), Gqq = c * conj(u);
                for (int k = 0; k < 5; ++k) { /* columns: A <- A G */
                    const cplx akp = A[k][p], akq = A[k][q];
                    A[k][p] = akp * Gpp + akq * Gqp;
                    A[k][q] = akp * Gpq + akq * Gqq;
                    const cplx qkp = Q[k][p], qkq = Q[k][q];
                    Q[k][p] = qkp * Gpp + qkq * Gqp;
                    Q[k][q] = qkp * Gpq + qkq * Gqq;
                }
                for (int k = 0; k < 5; ++k) { /* rows: A <- G^H A */
                    const cplx apk = A[p][k], aqk = A[q][k];
                    A[p][k] = conj(Gpp) * apk + conj(Gqp) * aqk;
                    A[q][k] = conj(Gpq) * apk + conj(Gqq) * aqk;
                }
                A[p][q] = 0.0;
                A[q][p] = 0.0;
                A[p][p] = creal(A[p][p]);
                A[q][q] = creal(A[q][q]);
            }
    }
    for (int i = 0; i < 5; ++i) lam[i] = creal(A[i][i]);
}

/* U = exp(-i delta V) = sum_k e^{-i delta lambda_k} v_k v_k^dagger (spectral theorem). */
static void expm_herm(const cplx V[5][5], double delta, cplx U[5][5]) {
    cplx A[5][5], Q[5][5];
    double lam[5];
    memcpy(A, V, sizeof(A));
    herm_eig(A, lam, Q);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < 5; ++k) acc += Q[i][k] * cexp(-I * delta * lam[k]) * conj(Q[j][k]);
            U[i][j] = acc;
        }
}

/* ---------------------------------------------------------------- potential step */

/* U = exp(-i delta V(psi)) at every site, psi = a + b, applied to the 5-vector a and to the
 * 5-vector b (Sec. VII.B; the operator itself is the plain-step factor U, or U^(1/4),
 * U^(1/8) of the interleaved step through delta). */
static void apply_potential(double* st, const oracle_cfg* cfg, double delta) {
    const long n = cfg->nx * cfg->ny;
#pragma omp parallel for schedule(static)
    for (long site = 0; site < n; ++site) {
        cplx a[5], b[5], psi[5], V[5][5], U[5][5];
        for (int m = 0; m < 5; ++m) {
            a[m] = getc(amp(st, n, m, site, 0));
            b[m] = getc(amp(st, n, m, site, 1));
            psi[m] = a[m] + b[m];
        }
        potential_matrix(psi, cfg->g0, cfg->g1, cfg->g2, V);
        expm_herm(V, delta, U);
        for (int i = 0; i < 5; ++i) {
            cplx ua = 0.0, ub = 0.0;
            for (int j = 0; j < 5; ++j) {
                ua += U[i][j] * a[j];
                ub += U[i][j] * b[j];
            }
            putc_(amp(st, n, i, site, 0), ua);
            putc_(amp(st, n, i, site, 1), ub);
        }
    }
}

/* ---------------------------------------------------------------- kinetic operator */

/* The 2x2 collide on every qubit pair (a_m, b_m).  which = 0: the collide C of the
 * variant; which = 1: the second collide of a block (C for K1, C^dagger for K2). */
static void collide_matrix(const oracle_cfg* cfg, int which, cplx C[2][2]) {
    if (cfg->kinetic_variant == 0 || which == 1) {
        C[0][0] = 0.5 * (1.0 - I); C[0][1] = 0.5 * (1.0 + I);
        C[1][0] = 0.5 * (1.0 + I); C[1][1] = 0.5 * (1.0 - I);
    } else {
        C[0][0] = 0.5 * (1.0 + I); C[0][1] = 0.5 * (1.0 - I);
        C[1][0] = 0.5 * (1.0 - I); C[1][1] = 0.5 * (1.0 + I);
    }
    /* K1 uses C twice; K2 uses C then C^dagger, and C_K2^dagger equals C_K1. */
}

/* adjoint = 1 applies the conjugate transpose of the collide instead. */
static void collide_any(double* st, const oracle_cfg* cfg, int which, int adjoint) {
    const long n = cfg->nx * cfg->ny;
    cplx C[2][2];
    collide_matrix(cfg, which, C);
    if (adjoint) {
        const cplx c01 = C[0][1];
        C[0][0] = conj(C[0][0]);
        C[1][1] = conj(C[1][1]);
        C[0][1] = conj(C[1][0]);
        C[1][0] = conj(c01);
    }
#pragma omp parallel for schedule(static)
    for (long site = 0; site < n; ++site)
        for (int m = 0; m < 5; ++m) {
            double* pa = amp(st, n, m, site, 0);
            double* pb = amp(st, n, m, site, 1);
            const cplx a = getc(pa), b = getc(pb);
            putc_(pa, C[0][0] * a + C[0][1] * b);
            putc_(pb, C[1][0] * a + C[1][1] * b);
        }
}

static void collide(double* st, const oracle_cfg* cfg, int which) { collide_any(st, cfg, which, 0); }

/* Stream qubit q of every level one site along `axis` (0 = x, 1 = y):
 * dir = +1 is S_q, q(j) <- q(j-1); dir = -1 is S^T_q, q(j) <- q(j+1).  Periodic. */
static void stream(double* st, const oracle_cfg* cfg, int axis, int q, int dir) {
    const long nx = cfg->nx, ny = cfg->ny, n = nx * ny;
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * n);
    for (int m = 0; m < 5; ++m) {
        for (long site = 0; site < n; ++site) tmp[site] = getc(amp(st, n, m, site, q));
#pragma omp parallel for schedule(static)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long sx = x, sy = y;
                if (axis == 0) sx = ((x - dir) % nx + nx) % nx;
                else sy = ((y - dir) % ny + ny) % ny;
                putc_(amp(st, n, m, y * nx + x, q), tmp[sy * nx + sx]);
            }
    }
    free(tmp);
}

/* One kinetic block I'_c = S_c C S^T_c C along `axis` for qubit c = q (operators act
 * right to left). */
static void kinetic_block(double* st, const oracle_cfg* cfg, int axis, int q) {
    collide(st, cfg, 0);
    stream(st, cfg, axis, q, -1);
    collide(st, cfg, 1);
    stream(st, cfg, axis, q, +1);
}

/* Block order on one axis: I'_1 I'_1 I'_2 I'_2 acting on psi, i.e. qubit 2 (b) twice, then
 * qubit 1 (a) twice. */
static const int block_qubit[4] = {1, 1, 0, 0};

static void apply_kinetic(double* st, const oracle_cfg* cfg) {
    for (int axis = 0; axis < cfg->ndim; ++axis)
        for (int k = 0; k < 4; ++k) kinetic_block(st, cfg, axis, block_qubit[k]);
}

/* ---------------------------------------------------------------- the time step */

/* Plain step psi(t+1) = K U psi(t); interleaved step: U^(1/4) (1D) or U^(1/8) (2D) before
 * every kinetic block, in the product order of the interleaved formula of Sec. VII.B. */
static void step_once(double* st, const oracle_cfg* cfg) {
    if (!cfg->interleave) {
        apply_potential(st, cfg, 1.0);
        apply_kinetic(st, cfg);
        return;
    }
    const double frac = 1.0 / (4.0 * cfg->ndim);
    for (int axis = 0; axis < cfg->ndim; ++axis)
        for (int k = 0; k < 4; ++k) {
            apply_potential(st, cfg, frac);
            kinetic_block(st, cfg, axis, block_qubit[k]);
        }
}

/* ---------------------------------------------------------------- adjoint (reverse mode)
 *
 * Pull-back of a cotangent through the plain step x' = K U(x) x (Sec. VII.B), for gradients of a
 * real loss L.  The cotangent of a complex amplitude z is gbar = dL/dRe z + i dL/dIm z, so that
 * dL = Re sum conj(gbar) dz; in the state layout it is stored like the state.
 *
 * Kinetic part.  K is complex-linear and unitary, so gbar_x = K^dagger gbar_x'.  K^dagger runs the
 * axes in reverse order (y, then x) and on each axis the blocks in reverse order; the adjoint of a
 * block S_c C' S^T_c C is C^dagger S_c C'^dagger S^T_c (S^T_c acts first).
 *
 * Potential part.  a' = U a, b' = U b with U = exp(A), A = -i delta V(psi), psi = a + b.  Then
 *   gbar_a = U^dagger gbar_a' + h,   gbar_b = U^dagger gbar_b' + h,
 * where h carries the dependence of V on psi.  With Mt = a gbar_a'^dagger + b gbar_b'^dagger, the
 * change of L through dU is Re tr(dU Mt); dU = L(A, dA) is the Frechet derivative of exp, and
 * tr(L(A, E) Mt) = tr(E L(A, Mt)), so with G = L(A, Mt) and the Hermitian H = (G - G^dagger)/(2i):
 *   dL = delta tr(dV H)   (dV Hermitian).
 * dV = g0 drho 1 + g1 sum_nu dF_nu f_nu + (g2/5)(ds s^dagger + s ds^dagger), drho = 2 Re psi^dagger dpsi,
 * dF_nu = 2 Re psi^dagger f_nu dpsi, ds = J conj(dpsi), give
 *   h = delta [2 g0 tr(H) psi + 2 g1 sum_nu tr(f_nu H) f_nu psi + (2 g2/5) J conj(H s)],
 * and the coupling gradients delta rho tr(H), delta sum_nu F_nu tr(f_nu H), (delta/5) s^dagger H s.
 * L(A, E) is taken in the eigenbasis of V (Daleckii-Krein): with V = Q diag(lambda) Q^dagger,
 * (Q^dagger L(A, E) Q)_ij = (Q^dagger E Q)_ij phi_ij, phi_ij the divided difference of
 * exp(-i delta lambda) at lambda_i, lambda_j: exp(-i delta (lambda_i + lambda_j)/2) sinc(delta
 * (lambda_i - lambda_j)/2), which is exp(-i delta lambda_i) when they coincide.
 */

static cplx divided_difference_exp(double li, double lj, double delta) {
    const double x = 0.5 * delta * (li - lj);
    const double sinc = (x == 0.0) ? 1.0 : sin(x) / x;
    return cexp(-I * delta * 0.5 * (li + lj)) * sinc;
}

/* L(-i delta V, E) for Hermitian V (the Frechet derivative of exp at A = -i delta V). */
static void frechet_exp_herm(const cplx V[5][5], double delta, const cplx E[5][5], cplx Lout[5][5]) {
    cplx A[5][5], Q[5][5], T[5][5], Et[5][5];
    double lam[5];
    memcpy(A, V, sizeof(A));
    herm_eig(A, lam, Q);
    for (int i = 0; i < 5; ++i) /* T = E Q */
        for (int j = 0; j < 5; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < 5; ++k) acc += E[i][k] * Q[k][j];
            T[i][j] = acc;
        }
    for (int i = 0; i < 5; ++i) /* Et = (Q^dagger E Q) o phi */
        for (int j = 0; j < 5; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < 5; ++k) acc += conj(Q[k][i]) * T[k][j];
            Et[i][j] = acc * divided_difference_exp(lam[i], lam[j], delta);
        }
    for (int i = 0; i < 5; ++i) /* T = Q Et */
        for (int j = 0; j < 5; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < 5; ++k) acc += Q[i][k] * Et[k][j];
            T[i][j] = acc;
        }
    for (int i = 0; i < 5; ++i) /* L = T Q^dagger */
        for (int j = 0; j < 5; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < 5; ++k) acc += T[i][k] * conj(Q[j][k]);
            Lout[i][j] = acc;
        }
}

/* The pull-back through U at one site: (ga, gb) hold the cotangents of (a', b') on entry and
 * those of (a, b) on exit; dcoup[3] accumulates dL/d(g0, g1, g2). */
static void potential_vjp_site(const cplx a[5], const cplx b[5], cplx ga[5], cplx gb[5],
                               const oracle_cfg* cfg, double delta, double dcoup[3]) {
    cplx psi[5], V[5][5], U[5][5], Mt[5][5], G[5][5], H[5][5];
    cplx fx[5][5], fy[5][5], fz[5][5];
    spin2_matrices(fx, fy, fz);
    cplx (*f[3])[5] = {fx, fy, fz};
    for (int m = 0; m < 5; ++m) psi[m] = a[m] + b[m];
    potential_matrix(psi, cfg->g0, cfg->g1, cfg->g2, V);
    expm_herm(V, delta, U);
    cplx pa[5], pb[5]; /* U^dagger applied to the incoming cotangents */
    for (int i = 0; i < 5; ++i) {
        pa[i] = 0.0;
        pb[i] = 0.0;
        for (int j = 0; j < 5; ++j) {
            pa[i] += conj(U[j][i]) * ga[j];
            pb[i] += conj(U[j][i]) * gb[j];
        }
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Mt[i][j] = a[i] * conj(ga[j]) + b[i] * conj(gb[j]);
    frechet_exp_herm(V, delta, Mt, G);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) H[i][j] = (G[i][j] - conj(G[j][i])) / (2.0 * I);
    double rho = 0.0, trH = 0.0, F[3], trfH[3];
    for (int i = 0; i < 5; ++i) {
        rho += creal(conj(psi[i]) * psi[i]);
        trH += creal(H[i][i]);
    }
    for (int nu = 0; nu < 3; ++nu) {
        cplx fv = 0.0, tr = 0.0;
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                fv += conj(psi[i]) * f[nu][i][j] * psi[j];
                tr += f[nu][i][j] * H[j][i];
            }
        F[nu] = creal(fv);
        trfH[nu] = creal(tr);
    }
    cplx s[5], Hs[5], sHs = 0.0;
    for (int i = 0; i < 5; ++i) {
        const int m = 2 - i;
        s[i] = ((m % 2 == 0) ? 1.0 : -1.0) * conj(psi[4 - i]);
    }
    for (int i = 0; i < 5; ++i) {
        Hs[i] = 0.0;
        for (int j = 0; j < 5; ++j) Hs[i] += H[i][j] * s[j];
    }
    for (int i = 0; i < 5; ++i) sHs += conj(s[i]) * Hs[i];
    for (int i = 0; i < 5; ++i) {
        cplx h = 2.0 * cfg->g0 * trH * psi[i];
        for (int nu = 0; nu < 3; ++nu)
            for (int j = 0; j < 5; ++j) h += 2.0 * cfg->g1 * trfH[nu] * f[nu][i][j] * psi[j];
        const int m = 2 - i;
        h += (2.0 * cfg->g2 / 5.0) * ((m % 2 == 0) ? 1.0 : -1.0) * conj(Hs[4 - i]);
        h *= delta;
        ga[i] = pa[i] + h;
        gb[i] = pb[i] + h;
    }
    dcoup[0] += delta * rho * trH;
    dcoup[1] += delta * (F[0] * trfH[0] + F[1] * trfH[1] + F[2] * trfH[2]);
    dcoup[2] += delta * creal(sHs) / 5.0;
}

/* st: the state x before U; cot: cotangent of U(x) x on entry, of x on exit. */
static void potential_vjp(const double* st, double* cot, const oracle_cfg* cfg, double delta,
                          double dcoup[3]) {
    const long n = cfg->nx * cfg->ny;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : d0, d1, d2)
    for (long site = 0; site < n; ++site) {
        cplx a[5], b[5], ga[5], gb[5];
        double dc[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < 5; ++m) {
            a[m] = getc(amp((double*)st, n, m, site, 0));
            b[m] = getc(amp((double*)st, n, m, site, 1));
            ga[m] = getc(amp(cot, n, m, site, 0));
            gb[m] = getc(amp(cot, n, m, site, 1));
        }
        potential_vjp_site(a, b, ga, gb, cfg, delta, dc);
        for (int m = 0; m < 5; ++m) {
            putc_(amp(cot, n, m, site, 0), ga[m]);
            putc_(amp(cot, n, m, site, 1), gb[m]);
        }
        d0 += dc[0];
        d1 += dc[1];
        d2 += dc[2];
    }
    dcoup[0] += d0;
    dcoup[1] += d1;
    dcoup[2] += d2;
}

/* K^dagger applied to a cotangent (or any field): axes, blocks and factors in reverse order,
 * each factor replaced by its adjoint. */
static void kinetic_block_adjoint(double* st, const oracle_cfg* cfg, int axis, int q) {
    stream(st, cfg, axis, q, -1);     /* (S_c)^dagger = S^T_c */
    collide_any(st, cfg, 1, 1);       /* C'^dagger */
    stream(st, cfg, axis, q, +1);     /* (S^T_c)^dagger = S_c */
    collide_any(st, cfg, 0, 1);       /* C^dagger */
}

static void apply_kinetic_adjoint(double* st, const oracle_cfg* cfg) {
    for (int axis = cfg->ndim - 1; axis >= 0; --axis)
        for (int k = 3; k >= 0; --k) kinetic_block_adjoint(st, cfg, axis, block_qubit[k]);
}

/* One plain step pulled back: cot <- (d step / d x)^T cot at the state x. */
static void vjp_step(const double* x, double* cot, const oracle_cfg* cfg, double dcoup[3]) {
    apply_kinetic_adjoint(cot, cfg);
    potential_vjp(x, cot, cfg, 1.0, dcoup);
}

/* ---------------------------------------------------------------- observables */

/* Sums over the lattice of the boson field psi = a + b (Sec. III.B Eq. cmap, Sec. IV.B Eq.
 * disecrete_energy); out[] order:
 *  0 norm_qubit  1 norm_boson  2..6 pop[m=+2..-2]  7 magnetisation  8 energy
 *  9 singlet_re  10 singlet_im  11 sum |psi^T J psi|^2  12 sum rho^2
 *  13 overlap_re  14 overlap_im
 * Energy density: sum_axis sum_m |psi_m(j+1) - psi_m(j)|^2 + g0/2 rho^2 + g1/2 |F|^2
 * + g2/10 |psi^T J psi|^2 (the functional whose variation gives V(psi) psi). */
static void observables(const double* st, const double* ref, const oracle_cfg* cfg,
                        double out[15]) {
    const long nx = cfg->nx, ny = cfg->ny, n = nx * ny;
    cplx fx[5][5], fy[5][5], fz[5][5];
    spin2_matrices(fx, fy, fz);
    for (int k = 0; k < 15; ++k) out[k] = 0.0;
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            const long site = y * nx + x;
            cplx psi[5];
            for (int m = 0; m < 5; ++m) {
                const cplx a = getc(amp((double*)st, n, m, site, 0));
                const cplx b = getc(amp((double*)st, n, m, site, 1));
                psi[m] = a + b;
                const double pm = creal(conj(a) * a) + creal(conj(b) * b);
                out[0] += pm;
                out[2 + m] += pm;
                out[7] += (2 - m) * pm;
            }
            double rho = 0.0;
            for (int m = 0; m < 5; ++m) rho += creal(conj(psi[m]) * psi[m]);
            out[1] += rho;
            double F2 = 0.0;
            cplx (*f[3])[5] = {fx, fy, fz};
            for (int nu = 0; nu < 3; ++nu) {
                cplx acc = 0.0;
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j < 5; ++j) acc += conj(psi[i]) * f[nu][i][j] * psi[j];
                F2 += creal(acc) * creal(acc);
            }
            cplx theta = 0.0; /* psi^T J psi = sum_m (-1)^m psi_m psi_{-m} */
            for (int i = 0; i < 5; ++i) {
                const int m = 2 - i;
                theta += ((m % 2 == 0) ? 1.0 : -1.0) * psi[i] * psi[4 - i];
            }
            const double th2 = creal(theta * conj(theta));
            double grad = 0.0;
            for (int axis = 0; axis < cfg->ndim; ++axis) {
                const long xn = axis == 0 ? (x + 1) % nx : x;
                const long yn = axis == 1 ? (y + 1) % ny : y;
                const long sn = yn * nx + xn;
                for (int m = 0; m < 5; ++m) {
                    const cplx pn = getc(amp((double*)st, n, m, sn, 0)) + getc(amp((double*)st, n, m, sn, 1));
                    const cplx d = pn - psi[m];
                    grad += creal(conj(d) * d);
                }
            }
            out[8] += grad + 0.5 * cfg->g0 * rho * rho + 0.5 * cfg->g1 * F2 + 0.1 * cfg->g2 * th2;
            out[9] += creal(theta) / sqrt(5.0);
            out[10] += cimag(theta) / sqrt(5.0);
            out[11] += th2;
            out[12] += rho * rho;
            if (ref) {
                for (int m = 0; m < 5; ++m) {
                    const cplx r = getc(amp((double*)ref, n, m, site, 0)) + getc(amp((double*)ref, n, m, site, 1));
                    const cplx ov = conj(psi[m]) * r;
                    out[13] += creal(ov);
                    out[14] += cimag(ov);
                }
            }
        }
}

/* ---------------------------------------------------------------- per-site fields */

/* Wrap a phase difference into (-pi, pi]. */
static double wrap_phase(double d) {
    while (d > kPi) d -= 2.0 * kPi;
    while (d <= -kPi) d += 2.0 * kPi;
    return d;
}

/* Per-site diagnostic fields of the boson field psi = a + b, 11 planes of nx*ny doubles:
 *  0 F_par = psi^dagger f_z psi            (Eq. cmap; the printed squares read as |psi_m|^2)
 *  1 F_perp = sqrt(F_x^2 + F_y^2)          (Eq. cmap, F_nu = psi^dagger f_nu psi)
 *  2 |A00| = |psi^T J psi| / sqrt(5)       (the singlet amplitude, Table II)
 *  3..5 (r, g, b) = (|F_par|, F_perp, |A00|) / their Euclidean norm, 0 where all vanish
 *       (Eq. colormap)
 *  6..10 vorticity of level m = +2..-2 (2D only, else 0): phase S = arg psi_m, central-difference
 *       velocity v_x = wrap(S(x+1) - S(x-1))/2, v_y likewise (Eq. velocity), and its
 *       central-difference curl (v_y(x+1) - v_y(x-1) - v_x(y+1) + v_x(y-1))/2 (the reading of
 *       Eq. pointwise_vorticity). */
static cplx boson_at(const double* st, long n, int m, long site) {
    return getc(amp((double*)st, n, m, site, 0)) + getc(amp((double*)st, n, m, site, 1));
}

static void fields(const double* st, const oracle_cfg* cfg, double* out) {
    const long nx = cfg->nx, ny = cfg->ny, n = nx * ny;
    cplx fx[5][5], fy[5][5], fz[5][5];
    spin2_matrices(fx, fy, fz);
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            const long site = y * nx + x;
            cplx psi[5];
            for (int m = 0; m < 5; ++m) psi[m] = boson_at(st, n, m, site);
            double F[3];
            cplx (*f[3])[5] = {fx, fy, fz};
            for (int nu = 0; nu < 3; ++nu) {
                cplx acc = 0.0;
                for (int i = 0; i < 5; ++i)
                    for (int j = 0; j < 5; ++j) acc += conj(psi[i]) * f[nu][i][j] * psi[j];
                F[nu] = creal(acc);
            }
            cplx theta = 0.0;
            for (int i = 0; i < 5; ++i) theta += (((2 - i) % 2 == 0) ? 1.0 : -1.0) * psi[i] * psi[4 - i];
            const double fpar = F[2], fperp = sqrt(F[0] * F[0] + F[1] * F[1]);
            const double a00 = cabs(theta) / sqrt(5.0);
            const double nrm = sqrt(fpar * fpar + fperp * fperp + a00 * a00);
            out[0 * n + site] = fpar;
            out[1 * n + site] = fperp;
            out[2 * n + site] = a00;
            out[3 * n + site] = nrm > 0 ? fabs(fpar) / nrm : 0.0;
            out[4 * n + site] = nrm > 0 ? fperp / nrm : 0.0;
            out[5 * n + site] = nrm > 0 ? a00 / nrm : 0.0;
            for (int m = 0; m < 5; ++m) {
                double w = 0.0;
                if (cfg->ndim == 2) {
                    const long xp = (x + 1) % nx, xm = (x + nx - 1) % nx;
                    const long yp = (y + 1) % ny, ym = (y + ny - 1) % ny;
                    const double Spp = carg(boson_at(st, n, m, yp * nx + xp));
                    const double Spm = carg(boson_at(st, n, m, ym * nx + xp));
                    const double Smp = carg(boson_at(st, n, m, yp * nx + xm));
                    const double Smm = carg(boson_at(st, n, m, ym * nx + xm));
                    const double vy_xp = wrap_phase(Spp - Spm) / 2.0;   /* v_y(x+1, y) */
                    const double vy_xm = wrap_phase(Smp - Smm) / 2.0;   /* v_y(x-1, y) */
                    const double vx_yp = wrap_phase(Spp - Smp) / 2.0;   /* v_x(x, y+1) */
                    const double vx_ym = wrap_phase(Spm - Smm) / 2.0;   /* v_x(x, y-1) */
                    w = (vy_xp - vy_xm - vx_yp + vx_ym) / 2.0;
                }
                out[(6 + m) * n + site] = w;
            }
        }
}

/* ---------------------------------------------------------------- exported entry points */

static int cfg_ok(const oracle_cfg* cfg) {
    if (!cfg) return 0;
    if (cfg->ndim != 1 && cfg->ndim != 2) return 0;
    if (cfg->nx < 1 || cfg->ny < 1) return 0;
    if (cfg->ndim == 1 && cfg->ny != 1) return 0;
    return 1;
}

int oracle_step(double* state, const oracle_cfg* cfg, long nsteps, int nthreads) {
    if (!cfg_ok(cfg) || !state || nsteps < 0) return 1;
    set_threads(nthreads);
    for (long s = 0; s < nsteps; ++s) step_once(state, cfg);
    return 0;
}

int oracle_apply_potential(double* state, const oracle_cfg* cfg, double delta, int nthreads) {
    if (!cfg_ok(cfg) || !state) return 1;
    set_threads(nthreads);
    apply_potential(state, cfg, delta);
    return 0;
}

int oracle_apply_kinetic(double* state, const oracle_cfg* cfg, int nthreads) {
    if (!cfg_ok(cfg) || !state) return 1;
    set_threads(nthreads);
    apply_kinetic(state, cfg);
    return 0;
}

/* Single operators for the tests: which = 0 collide C, 1 second collide, 2 stream. */
int oracle_apply_operator(double* state, const oracle_cfg* cfg, int which, int axis, int q,
                          int dir) {
    if (!cfg_ok(cfg) || !state) return 1;
    if (which == 0 || which == 1) collide(state, cfg, which);
    else if (which == 2) stream(state, cfg, axis, q, dir);
    else return 1;
    return 0;
}

int oracle_observables(const double* state, const double* ref, const oracle_cfg* cfg,
                       double* out15) {
    if (!cfg_ok(cfg) || !state || !out15) return 1;
    observables(state, ref, cfg, out15);
    return 0;
}

/* psi10 = (re, im) of psi_{+2..-2}; V50 = 5x5 complex row-major (re, im). */
int oracle_potential_matrix(const double* psi10, double g0, double g1, double g2, double* V50) {
    cplx psi[5], V[5][5];
    for (int i = 0; i < 5; ++i) psi[i] = psi10[2 * i] + I * psi10[2 * i + 1];
    potential_matrix(psi, g0, g1, g2, V);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            V50[2 * (5 * i + j)] = creal(V[i][j]);
            V50[2 * (5 * i + j) + 1] = cimag(V[i][j]);
        }
    return 0;
}

/* Hermitian eigendecomposition of V50: lam5 ascending order not guaranteed; Q50 columns. */
int oracle_heig(const double* V50, double* lam5, double* Q50) {
    cplx A[5][5], Q[5][5];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) A[i][j] = V50[2 * (5 * i + j)] + I * V50[2 * (5 * i + j) + 1];
    herm_eig(A, lam5, Q);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            Q50[2 * (5 * i + j)] = creal(Q[i][j]);
            Q50[2 * (5 * i + j) + 1] = cimag(Q[i][j]);
        }
    return 0;
}

int oracle_expm(const double* V50, double delta, double* U50) {
    cplx V[5][5], U[5][5];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) V[i][j] = V50[2 * (5 * i + j)] + I * V50[2 * (5 * i + j) + 1];
    expm_herm(V, delta, U);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            U50[2 * (5 * i + j)] = creal(U[i][j]);
            U50[2 * (5 * i + j) + 1] = cimag(U[i][j]);
        }
    return 0;
}

int oracle_fields(const double* state, const oracle_cfg* cfg, double* out11) {
    if (!cfg_ok(cfg) || !state || !out11) return 1;
    fields(state, cfg, out11);
    return 0;
}

/* Adjoint entry points (plain step only; the interleaved step returns 2).
 * oracle_vjp_potential: cot (cotangent of U(x) x) -> cotangent of x at state x, with delta.
 * oracle_vjp_kinetic:   field <- K^dagger field.
 * oracle_vjp_step:      cot (cotangent of step(x)) -> cotangent of x.
 * oracle_vjp_run:       forward nsteps from x0 keeping every state, then pull cot (cotangent of
 *                       the final state) back to the cotangent of x0.
 * dcoup3 accumulates dL/d(g0, g1, g2). */
int oracle_vjp_potential(const double* x, double* cot, const oracle_cfg* cfg, double delta,
                         double* dcoup3, int nthreads) {
    if (!cfg_ok(cfg) || !x || !cot || !dcoup3) return 1;
    set_threads(nthreads);
    potential_vjp(x, cot, cfg, delta, dcoup3);
    return 0;
}

int oracle_vjp_kinetic(double* field, const oracle_cfg* cfg, int nthreads) {
    if (!cfg_ok(cfg) || !field) return 1;
    set_threads(nthreads);
    apply_kinetic_adjoint(field, cfg);
    return 0;
}

int oracle_vjp_step(const double* x, double* cot, const oracle_cfg* cfg, double* dcoup3, int nthreads) {
    if (!cfg_ok(cfg) || !x || !cot || !dcoup3) return 1;
    if (cfg->interleave) return 2;
    set_threads(nthreads);
    vjp_step(x, cot, cfg, dcoup3);
    return 0;
}

int oracle_vjp_run(const double* x0, long nsteps, double* cot, const oracle_cfg* cfg,
                   double* dcoup3, int nthreads) {
    if (!cfg_ok(cfg) || !x0 || !cot || !dcoup3 || nsteps < 0) return 1;
    if (cfg->interleave) return 2;
    set_threads(nthreads);
    const size_t len = (size_t)(cfg->nx * cfg->ny) * 20;
    double* hist = (double*)malloc(sizeof(double) * len * (size_t)(nsteps > 0 ? nsteps : 1));
    if (!hist) return 3;
    if (nsteps > 0) memcpy(hist, x0, sizeof(double) * len);
    for (long k = 1; k < nsteps; ++k) {
        memcpy(hist + k * len, hist + (k - 1) * len, sizeof(double) * len);
        step_once(hist + k * len, cfg);
    }
    for (long k = nsteps - 1; k >= 0; --k) vjp_step(hist + k * len, cot, cfg, dcoup3);
    free(hist);
    return 0;
}

/* L(-i delta V, E) for Hermitian V; V50, E50, L50: 5x5 complex row-major (re, im). */
int oracle_frechet_exp(const double* V50, double delta, const double* E50, double* L50) {
    cplx V[5][5], E[5][5], Lm[5][5];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            V[i][j] = V50[2 * (5 * i + j)] + I * V50[2 * (5 * i + j) + 1];
            E[i][j] = E50[2 * (5 * i + j)] + I * E50[2 * (5 * i + j) + 1];
        }
    frechet_exp_herm(V, delta, E, Lm);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            L50[2 * (5 * i + j)] = creal(Lm[i][j]);
            L50[2 * (5 * i + j) + 1] = cimag(Lm[i][j]);
        }
    return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
