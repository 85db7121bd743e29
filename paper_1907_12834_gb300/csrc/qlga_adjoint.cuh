// qlga_adjoint.cuh -- reverse mode (adjoint) of the plain QLGA step (arXiv:1907.12834, Sec. VII.B).
//
// For a real loss L of the state, the cotangent of a complex amplitude z is gbar = dL/dRe z +
// i dL/dIm z (so dL = Re sum conj(gbar) dz); a cotangent buffer has the state's layout.  One
// plain step x' = K U(x) x pulls a cotangent back as
//   gbar_x = U_x^T (K^dagger gbar_x')
// where K^dagger is the adjoint kinetic operator (axes, blocks and factors in reverse order, each
// factor replaced by its adjoint) and U_x^T the transposed linearisation of the potential step at
// the state x, which includes the dependence of V on psi.
//
// Potential step at one site (a' = U a, b' = U b, U = exp(-i delta V(psi)), psi = a + b):
//   gbar_a = U^dagger gbar_a' + h,   gbar_b = U^dagger gbar_b' + h,
// with h the gradient through psi.  Writing V = c 1 + W (c = (g0 + g2/10) rho) and B = -i delta W,
// U = e^{-i delta c} P(B) with P the Taylor polynomial of the forward step.  With
// M = a gbar_a'^dagger + b gbar_b'^dagger and the Frechet derivative L(B, E) = d/dt P(B + t E):
//   tau    = Im tr(U M) = Im sum_r gbar_r^dagger U x_r                        (r = a, b)
//   phi_nu = Im tr(f_nu G),  G = e^{-i delta c} L(B, M),  tr(f_nu G) = e^{-i delta c} sum_r
//            gbar_r^dagger L(B, f_nu) x_r                                      (nu = x, y, z)
//   H s    = (G s - G^dagger s) / (2i),  s = J conj(psi),
//            G s = e^{-i delta c} L(B, M) s,  G^dagger s = e^{i delta c} L(-B, M^dagger) s
//   h      = delta [2 g0 tau psi + 2 g1 sum_nu phi_nu f_nu psi + (2 g2/5) J conj(H s)]
// and the coupling gradients dL/dg0 = delta rho tau, dL/dg1 = delta sum_nu F_nu phi_nu,
// dL/dg2 = (delta/5) Re s^dagger H s.  (The identity direction of dV commutes with B; its
// derivative uses the exact exponential, whose trace form is tau.)
//
// Each L(B, E) v is the upper block of P([[B, E], [0, B]]) applied to (0, v): the same Horner
// recursion as the forward step on a pair of 5-vectors, with the degree the forward step used at
// that site.  No matrix is formed; everything is matrix-vector work on the tridiagonal-plus-
// rank-one W.
#pragma once

#include "qlga_device.cuh"

namespace qlga {

// ------------------------------------------------------------------ adjoint kinetic stencil
//
// K^dagger of one axis: the blocks' adjoints in reverse order.  A block I'_c = S_c C' S^T_c C has
// adjoint C^dagger S_c C'^dagger S^T_c (S^T_c acts first).  In the (a, bt) basis the real parts
// of the collides' adjoints are [[1, -1], [1, 1]] (adjoint of [[1, 1], [-1, 1]]) and vice versa;
// their scalar prefactors multiply to exactly 1/16 per axis, as for K.  Derived at compile time
// from the block definition on a unit impulse, like the forward table.
constexpr KinStencil make_stencil_adjoint(int variant) {
    KinStencil S{};
    const int block_qubit_rev[4] = {0, 0, 1, 1};
    for (int src = 0; src < 2; ++src) {
        int v[2][11] = {};
        v[src][5] = 1;
        for (int blk = 0; blk < 4; ++blk) {
            const int c = block_qubit_rev[blk];
            shift_int(v, c, -1);          // (S_c)^dagger = S^T_c
            collide_int(v, 1, -1, 1, 1);  // C'^dagger (C' is [[1, 1], [-1, 1]] in both variants)
            shift_int(v, c, +1);          // (S^T_c)^dagger = S_c
            if (variant == 0) collide_int(v, 1, -1, 1, 1);  // C^dagger, K1
            else collide_int(v, 1, 1, -1, 1);               // C^dagger, K2
        }
        for (int dst = 0; dst < 2; ++dst)
            for (int k = -4; k <= 4; ++k) S.g[dst][src][k + 4] = v[dst][5 - k];
    }
    return S;
}

constexpr KinStencil kStencilAdj[2] = {make_stencil_adjoint(0), make_stencil_adjoint(1)};

// ------------------------------------------------------------------ per-site pull-back of U

template <class T>
struct AdjConst {
    PotConst<T> pc;  // the forward step's constants (delta folded in)
    T dg0;           // delta g0
    T dg1;           // delta g1
    T dg2_5;         // delta g2 / 5
    T delta;
    AdjConst() = default;
    __host__ __device__ explicit AdjConst(const PotParams& P)
        : pc(P), dg0(T(P.delta * P.g0)), dg1(T(P.delta * P.g1)), dg2_5(T(P.delta * P.g2 / 5.0)),
          delta(T(P.delta)) {}
};

// Spin matrices of Sec. II on a 5-vector (rows m = +2..-2): off-diagonal entries c_i of f_x at
// (i, i+1) and (i+1, i); f_y has -i c_i and +i c_i there; f_z = diag(2, 1, 0, -1, -2).
template <class T>
__device__ __forceinline__ T spin_c(int i) {
    return (i == 0 || i == 3) ? T(1) : T(1.2247448713915890491);  // 1, sqrt(3/2), sqrt(3/2), 1
}

template <class T>
__device__ __forceinline__ void apply_fz(const cpx<T> x[5], cpx<T> y[5]) {
#pragma unroll
    for (int i = 0; i < 5; ++i) y[i] = T(2 - i) * x[i];
}
template <class T>
__device__ __forceinline__ void apply_fx(const cpx<T> x[5], cpx<T> y[5]) {
#pragma unroll
    for (int i = 0; i < 5; ++i) y[i] = {T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T c = spin_c<T>(i);
        y[i] = y[i] + c * x[i + 1];
        y[i + 1] = y[i + 1] + c * x[i];
    }
}
template <class T>
__device__ __forceinline__ void apply_fy(const cpx<T> x[5], cpx<T> y[5]) {
#pragma unroll
    for (int i = 0; i < 5; ++i) y[i] = {T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T c = spin_c<T>(i);
        // y_i += -i c x_{i+1};  y_{i+1} += i c x_i
        y[i] = {y[i].re + c * x[i + 1].im, y[i].im - c * x[i + 1].re};
        y[i + 1] = {y[i + 1].re - c * x[i].im, y[i + 1].im + c * x[i].re};
    }
}

// conj(x) . y
template <class T>
__device__ __forceinline__ cpx<T> cdot(const cpx<T> x[5], const cpx<T> y[5]) {
    cpx<T> acc = cmulc(x[0], y[0]);
#pragma unroll
    for (int i = 1; i < 5; ++i) acc = cfmac(x[i], y[i], acc);
    return acc;
}

// v = x + sgn * (-i) * ik * w   (one Horner step of P(sgn B) with B v = -i W v)
template <class T>
__device__ __forceinline__ void horner_sgn(const cpx<T> x[5], const cpx<T> w[5], cpx<T> v[5], T ik) {
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = {fma(ik, w[i].im, x[i].re), fma(-ik, w[i].re, x[i].im)};
}

// v = ik * (-i * w + e)  (upper block of the augmented Horner step); sik = sgn * ik
template <class T>
__device__ __forceinline__ void horner_upper(const cpx<T> w[5], const cpx<T> e[5], cpx<T> v[5], T sik,
                                             T ik) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
        v[i] = {fma(sik, w[i].im, ik * e[i].re), fma(-sik, w[i].re, ik * e[i].im)};
}

// The forward step's W at a site (as potential_site builds it, unscaled input) and its degree.
template <class T>
__device__ __forceinline__ int build_w(const cpx<T> psi[5], const PotConst<T>& C, WOp<T>& W, T& rho,
                                       T& Fz, cpx<T>& Fp, unsigned* status, T* beta_out = nullptr) {
    T n[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) n[i] = norm2(psi[i]);
    rho = (n[0] + n[1]) + (n[2] + n[3]) + n[4];
    Fz = T(2) * (n[0] - n[4]) + (n[1] - n[3]);
    const T r32 = T(1.2247448713915890491);
    Fp = cmulc(psi[0], psi[1]);
    Fp = cfmac(psi[3], psi[4], Fp);
    cpx<T> mid = cmulc(psi[1], psi[2]);
    mid = cfmac(psi[2], psi[3], mid);
    Fp = {fma(r32, mid.re, Fp.re), fma(r32, mid.im, Fp.im)};
    Fp = T(2) * Fp;
    const T Fabs = sqrt(fma(Fz, Fz, norm2(Fp)));
    const T beta = fma(C.b1, Fabs, C.b2 * rho);
    if (!(beta <= T(kBetaMax))) atomicOr(status, 1u);
    if (beta_out) *beta_out = beta;
    const int K = warp_taylor_degree(beta, TaylorTol<T>::value);
    const T g2r = C.dr * rho;
    const T gz = C.dz * Fz;
    W.D[0] = T(2) * gz - g2r;
    W.D[1] = gz - g2r;
    W.D[2] = -g2r;
    W.D[3] = -gz - g2r;
    W.D[4] = T(-2) * gz - g2r;
    W.ep[0] = C.e0 * Fp;
    W.ep[1] = C.e1 * Fp;
    W.ep[2] = W.ep[1];
    W.ep[3] = W.ep[0];
    W.u[0] = psi[4];
    W.u[1] = {-psi[3].re, -psi[3].im};
    W.u[2] = psi[2];
    W.u[3] = {-psi[1].re, -psi[1].im};
    W.u[4] = psi[0];
    W.R = C.R;
    return K;
}

// FP64 pull-backs run the Horner steps of order above k0 in FP32 (Kin = K - k0 inner steps) and
// the k0 outer ones in FP64, as the forward step does (zframe_inner_fp32), with k0 the smallest
// order whose bound beta^k0 / k0! is at most kAdjInnerTol: smaller than the forward's 2^-31
// because an error in the inner iterate of the lower recursion enters the Frechet terms once per
// outer step, multiplied by the spin or rank-two matrix (a factor up to ~k0 / beta more).
constexpr double kAdjInnerTol = 3.637978807091713e-12;  // 2^-38

template <class U>
__device__ __forceinline__ cpx<U> to_prec(cpx<double> z) { return {U(z.re), U(z.im)}; }

template <class U>
__device__ __forceinline__ WOp<U> wop_to(const WOp<double>& W) {
    WOp<U> V;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        V.D[i] = U(W.D[i]);
        V.u[i] = to_prec<U>(W.u[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) V.ep[i] = to_prec<U>(W.ep[i]);
    V.R = U(W.R);
    return V;
}

// One Horner step (1/k = ik) of trace_terms' four recursions.
template <class U>
__device__ __forceinline__ void trace_step(const WOp<U>& W, const cpx<U> x[5], cpx<U> v2[5], cpx<U> vx[5],
                                           cpx<U> vy[5], cpx<U> vz[5], U ik) {
    cpx<U> w[5], e[5];
    W.apply(vx, w);
    apply_fx(v2, e);
    horner_upper(w, e, vx, ik, ik);
    W.apply(vy, w);
    apply_fy(v2, e);
    horner_upper(w, e, vy, ik, ik);
    W.apply(vz, w);
    apply_fz(v2, e);
    horner_upper(w, e, vz, ik, ik);
    W.apply(v2, w);
    horner_sgn(x, w, v2, ik);
}

// tr terms of one input vector x_r with its output cotangent g_r:
//   tr_xyz[nu] += g_r^dagger L(B, f_nu) x_r,  tuc += g_r^dagger P(B) x_r
// Wf: W in FP32, for the Kin inner steps of an FP64 call.
template <class T>
__device__ __forceinline__ void trace_terms(const WOp<T>& W, const WOp<float>& Wf, const cpx<T> x[5],
                                            const cpx<T> g[5], int K, int Kin, cpx<T> tr[3], cpx<T>& tuc) {
    cpx<T> v2[5], vx[5], vy[5], vz[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        v2[i] = x[i];
        vx[i] = vy[i] = vz[i] = {T(0), T(0)};
    }
    int k = K;
    if constexpr (std::is_same<T, double>::value) {
        if (Kin > 0) {  // warp-uniform
            cpx<float> xf[5], v2f[5], vxf[5], vyf[5], vzf[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                xf[i] = to_prec<float>(x[i]);
                v2f[i] = xf[i];
                vxf[i] = vyf[i] = vzf[i] = {0.f, 0.f};
            }
            for (; k > K - Kin; --k) trace_step<float>(Wf, xf, v2f, vxf, vyf, vzf, inv_k(k, 0.f));
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                v2[i] = {double(v2f[i].re), double(v2f[i].im)};
                vx[i] = {double(vxf[i].re), double(vxf[i].im)};
                vy[i] = {double(vyf[i].re), double(vyf[i].im)};
                vz[i] = {double(vzf[i].re), double(vzf[i].im)};
            }
        }
    }
    for (; k >= 1; --k) trace_step<T>(W, x, v2, vx, vy, vz, inv_k(k, T(0)));
    tr[0] = tr[0] + cdot(g, vx);
    tr[1] = tr[1] + cdot(g, vy);
    tr[2] = tr[2] + cdot(g, vz);
    tuc = tuc + cdot(g, v2);
}

// One Horner step (1/k = ik) of frechet_rank2's two recursions.
template <class U>
__device__ __forceinline__ void frechet_step(const WOp<U>& W, const cpx<U> s[5], const cpx<U> p0[5],
                                             const cpx<U> q0[5], const cpx<U> p1[5], const cpx<U> q1[5],
                                             cpx<U> v2[5], cpx<U> out[5], U sgn, U ik) {
    cpx<U> w[5], e[5];
    const cpx<U> c0 = cdot(q0, v2), c1 = cdot(q1, v2);
#pragma unroll
    for (int i = 0; i < 5; ++i) e[i] = cfma(c1, p1[i], cmul(c0, p0[i]));
    W.apply(out, w);
    horner_upper(w, e, out, sgn * ik, ik);
    W.apply(v2, w);
    horner_sgn(s, w, v2, sgn * ik);
}

// q = L(sgn B, E) s with E v = sum_r p_r (q_r^dagger v): for G s take (p, q) = (x, g) and
// sgn = +1; for G^dagger s take (p, q) = (g, x) and sgn = -1.  Wf, Kin as in trace_terms.
template <class T>
__device__ __forceinline__ void frechet_rank2(const WOp<T>& W, const WOp<float>& Wf, const cpx<T> s[5],
                                              const cpx<T> p0[5], const cpx<T> q0[5], const cpx<T> p1[5],
                                              const cpx<T> q1[5], int K, int Kin, T sgn, cpx<T> out[5]) {
    cpx<T> v2[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        v2[i] = s[i];
        out[i] = {T(0), T(0)};
    }
    int k = K;
    if constexpr (std::is_same<T, double>::value) {
        if (Kin > 0) {  // warp-uniform
            cpx<float> sf[5], p0f[5], q0f[5], p1f[5], q1f[5], v2f[5], outf[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                sf[i] = to_prec<float>(s[i]);
                p0f[i] = to_prec<float>(p0[i]);
                q0f[i] = to_prec<float>(q0[i]);
                p1f[i] = to_prec<float>(p1[i]);
                q1f[i] = to_prec<float>(q1[i]);
                v2f[i] = sf[i];
                outf[i] = {0.f, 0.f};
            }
            for (; k > K - Kin; --k)
                frechet_step<float>(Wf, sf, p0f, q0f, p1f, q1f, v2f, outf, float(sgn), inv_k(k, 0.f));
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                v2[i] = {double(v2f[i].re), double(v2f[i].im)};
                out[i] = {double(outf[i].re), double(outf[i].im)};
            }
        }
    }
    for (; k >= 1; --k) frechet_step<T>(W, s, p0, q0, p1, q1, v2, out, sgn, inv_k(k, T(0)));
}

// Pull-back through U at one site.  (a, b): the state before U.  (ga, gb): cotangents of the
// outputs on entry, of the inputs on exit.  dc[3] = this site's dL/d(g0, g1, g2).
template <class T>
__device__ __forceinline__ void potential_vjp_site(const cpx<T> a[5], const cpx<T> b[5], cpx<T> ga[5],
                                                   cpx<T> gb[5], const AdjConst<T>& A, T dc[3],
                                                   unsigned* status) {
    cpx<T> psi[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) psi[i] = a[i] + b[i];
    WOp<T> W;
    T rho, Fz, beta;
    cpx<T> Fp;
    const int K = build_w(psi, A.pc, W, rho, Fz, Fp, status, &beta);
    int Kin = 0;  // FP64: inner Horner steps in FP32 (kAdjInnerTol)
    WOp<float> Wf;
    if constexpr (std::is_same<T, double>::value) {
        const int k0 = warp_max_int(taylor_degree(beta, kAdjInnerTol) + 1);
        Kin = K > k0 ? K - k0 : 0;
        Wf = wop_to<float>(W);
    }
    T sn, cs;
    sin_cos(A.pc.cphase * rho, &sn, &cs);
    const cpx<T> ph = {cs, -sn};  // e^{-i delta c}

    // tau and phi_nu
    cpx<T> tr[3] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    cpx<T> tuc = {T(0), T(0)};
    trace_terms(W, Wf, a, ga, K, Kin, tr, tuc);
    trace_terms(W, Wf, b, gb, K, Kin, tr, tuc);
    const T tau = cmul(ph, tuc).im;
    const T phx = cmul(ph, tr[0]).im, phy = cmul(ph, tr[1]).im, phz = cmul(ph, tr[2]).im;

    // H s
    cpx<T> s[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) s[i] = {W.u[i].re, -W.u[i].im};  // s = conj(u)
    cpx<T> q1[5], q2[5];
    frechet_rank2(W, Wf, s, a, ga, b, gb, K, Kin, T(1), q1);
    frechet_rank2(W, Wf, s, ga, a, gb, b, K, Kin, T(-1), q2);
    cpx<T> Hs[5];
    const cpx<T> phc = {cs, sn};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const cpx<T> d = cmul(ph, q1[i]) - cmul(phc, q2[i]);
        Hs[i] = {T(0.5) * d.im, T(-0.5) * d.re};  // d / (2i)
    }

    // h = 2 dg0 tau psi + 2 dg1 (phi_z f_z + phi_x f_x + phi_y f_y) psi + 2 dg2/5 J conj(H s)
    cpx<T> h[5], fpsi[5];
    const T t0 = T(2) * A.dg0 * tau;
#pragma unroll
    for (int i = 0; i < 5; ++i) h[i] = t0 * psi[i];
    const T t1 = T(2) * A.dg1;
    apply_fz(psi, fpsi);
#pragma unroll
    for (int i = 0; i < 5; ++i) h[i] = h[i] + (t1 * phz) * fpsi[i];
    apply_fx(psi, fpsi);
#pragma unroll
    for (int i = 0; i < 5; ++i) h[i] = h[i] + (t1 * phx) * fpsi[i];
    apply_fy(psi, fpsi);
#pragma unroll
    for (int i = 0; i < 5; ++i) h[i] = h[i] + (t1 * phy) * fpsi[i];
    const T t2 = T(2) * A.dg2_5;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const T sg = (i & 1) ? T(-1) : T(1);  // (-1)^m, m = 2 - i
        const cpx<T> c = {Hs[4 - i].re, -Hs[4 - i].im};
        h[i] = h[i] + (sg * t2) * c;
    }

    // coupling gradients
    cpx<T> sHs = {T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 5; ++i) sHs = cfma(W.u[i], Hs[i], sHs);  // conj(s_i) = u_i
    dc[0] = A.delta * rho * tau;
    dc[1] = A.delta * (Fp.re * phx + Fp.im * phy + Fz * phz);
    dc[2] = A.delta * sHs.re / T(5);

    // U^dagger on the incoming cotangents, plus h
    cpx<T> pa[5], pb[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        pa[i] = ga[i];
        pb[i] = gb[i];
    }
    int k = K;
    if constexpr (std::is_same<T, double>::value) {
        if (Kin > 0) {  // warp-uniform
            cpx<float> gaf[5], gbf[5], paf[5], pbf[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                gaf[i] = paf[i] = to_prec<float>(ga[i]);
                gbf[i] = pbf[i] = to_prec<float>(gb[i]);
            }
            for (; k > K - Kin; --k) {
                const float ik = inv_k(k, 0.f);
                cpx<float> wa[5], wb[5];
                Wf.apply(paf, wa);
                Wf.apply(pbf, wb);
                horner_sgn(gaf, wa, paf, -ik);
                horner_sgn(gbf, wb, pbf, -ik);
            }
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                pa[i] = {double(paf[i].re), double(paf[i].im)};
                pb[i] = {double(pbf[i].re), double(pbf[i].im)};
            }
        }
    }
    for (; k >= 1; --k) {
        const T ik = inv_k(k, T(0));
        cpx<T> wa[5], wb[5];
        W.apply(pa, wa);
        W.apply(pb, wb);
        horner_sgn(ga, wa, pa, -ik);
        horner_sgn(gb, wb, pb, -ik);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ga[i] = cmul(phc, pa[i]) + h[i];
        gb[i] = cmul(phc, pb[i]) + h[i];
    }
}

// ------------------------------------------------------------------ kernel

constexpr int kAdjThreads = 128;

// Per-thread sum of the per-site coupling-gradient terms: FP64 for an FP64 state; compensated
// (Kahan) FP32 for an FP32 state, whose terms carry FP32 rounding anyway and whose FP64 additions
// would cost 64 FP32 slots each.  Block sums are FP64.
template <class T>
struct AdjSum;
template <>
struct AdjSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct AdjSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) - double(c); }
};

// Resident pair (a, bt) of level m at a site.
template <class T>
__device__ __forceinline__ void load_resident(const T* X, int64_t nsites, int m, int64_t site, cpx<T>& a,
                                              cpx<T>& bt) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(X) + m * nsites + site);
        a = {v.x, v.y};
        bt = {v.z, v.w};
    } else {
        const double2* p = reinterpret_cast<const double2*>(X) + 2 * (m * nsites + site);
        const double2 u = __ldg(p), w = __ldg(p + 1);
        a = {u.x, u.y};
        bt = {w.x, w.y};
    }
}

// gout = [U_X^T o] K_axis^dagger gin on resident cotangent buffers: the adjoint nine-point
// stencil of one axis, optionally followed by the pull-back through U at the state X (resident,
// the true state before U).  VJP: dL/dg of this launch is added to partials[block][3] (each block
// owns its row, so repeated launches with the same grid accumulate deterministically).
template <class T, int VARIANT, bool VJP>
// FP32: 4 resident CTAs per SM (128 registers, a few spilled) beat 3 at 168 registers by 12%.
__global__ void __launch_bounds__(kAdjThreads, sizeof(T) == 4 ? 4 : 1) k_adjoint_axis(const T* __restrict__ gin, T* __restrict__ gout,
                                                              const T* __restrict__ X, int64_t nx, int64_t ny,
                                                              int axis, AdjConst<T> A,
                                                              double* __restrict__ partials, unsigned* status) {
    constexpr KinStencil S = kStencilAdj[VARIANT];
    const int64_t nsites = nx * ny;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    AdjSum<T> dsum[3];
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < nsites; base += stride) {
        const int64_t site = base + threadIdx.x;
        const bool active = site < nsites;
        const int64_t s = active ? site : 0;
        const int64_t x = s % nx, y = s / nx;
        int64_t nb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (axis == 0) {
                int64_t xx = x + k - 4;
                xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
                nb[k] = y * nx + xx;
            } else {
                int64_t yy = y + k - 4;
                yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
                nb[k] = yy * nx + x;
            }
        }
        cpx<T> ga[5], gb[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            cpx<T> acc_a = {T(0), T(0)}, acc_bt = {T(0), T(0)};
            static_for<9>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                cpx<T> a, bt;
                load_resident(gin, nsites, m, nb[k], a, bt);
                kin_tap4<S.g[0][0][k], S.g[0][1][k], S.g[1][0][k], S.g[1][1][k]>(a, bt, acc_a, acc_bt);
            });
            const T sc = T(0.0625);
            ga[m] = {sc * acc_a.re, sc * acc_a.im};
            gb[m] = {sc * acc_bt.im, -sc * acc_bt.re};  // b = -i bt
        }
        if (VJP) {
            cpx<T> a[5], b[5];
            SiteIO<T>::load(X, nsites, s, a, b);
            T dc[3];
            potential_vjp_site(a, b, ga, gb, A, dc, status);
            if (active) {
                dsum[0].add(dc[0]);
                dsum[1].add(dc[1]);
                dsum[2].add(dc[2]);
            }
        }
        if (active) SiteIO<T>::store(gout, nsites, site, ga, gb);
    }
    if (VJP) {
        __shared__ double sh[kAdjThreads / 32][3];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double v = dsum[j].value();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sh[wid][j] = v;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = 0.0;
            for (int w = 0; w < kAdjThreads / 32; ++w) v += sh[w][threadIdx.x];
            partials[int64_t(blockIdx.x) * 3 + threadIdx.x] += v;
        }
    }
}

}  // namespace qlga
