// qlga_device.cuh -- device building blocks of the spin-2 QLGA step (arXiv:1907.12834).
//
// Conventions shared by every kernel of the library:
//  * Resident state: 5 planes (m = +2..-2) of ny*nx sites, x fastest; a site is the qubit pair
//    of that level as (a.re, a.im, bt.re, bt.im) with bt = i*b.  One float4 (FP32) or two double2
//    (FP64) per site and plane, so a warp reading 32 consecutive sites of a plane reads 512 or
//    1024 contiguous bytes.  The C ABI's layout (a.re, a.im, b.re, b.im) is converted on load and
//    read-out only; SiteIO / load_pair return (a, b).  A 2D FP32 state held pending K for the
//    fused step is stored as (P, Q) = (a + bt, a - bt) instead (qlga_step2d.cuh): its x stencil
//    has fewer taps in that basis.
//  * Inside the kinetic operator the pair is carried as (a, bt) with bt = i*b.  In that basis the
//    collide C = 1/2 [[1-i, 1+i], [1+i, 1-i]] of a kinetic block (Sec. VII.B) becomes the scalar
//    (1-i)/2 times the real matrix [[1, 1], [-1, 1]], so a collide costs four real additions per
//    level.  The scalars of the eight collides of one axis multiply to exactly 1/16 (a power of
//    two), which is applied once, exactly, at the end.
#pragma once

#include <cstdint>
#include <limits>
#include <type_traits>
#include <cuda_runtime.h>

namespace qlga {

// ------------------------------------------------------------------ complex helpers

template <class T>
struct cpx {
    T re, im;
};

template <class T>
__device__ __forceinline__ cpx<T> mk(T r, T i) { return cpx<T>{r, i}; }
template <class T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T>
__device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
// a * b
template <class T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc + a * b
template <class T>
__device__ __forceinline__ cpx<T> cfma(cpx<T> a, cpx<T> b, cpx<T> acc) {
    return {fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im))};
}
// acc + conj(a) * b
template <class T>
__device__ __forceinline__ cpx<T> cfmac(cpx<T> a, cpx<T> b, cpx<T> acc) {
    return {fma(a.re, b.re, fma(a.im, b.im, acc.re)), fma(a.re, b.im, fma(-a.im, b.re, acc.im))};
}
template <class T>
__device__ __forceinline__ T norm2(cpx<T> a) { return fma(a.re, a.re, a.im * a.im); }

// ------------------------------------------------------------------ site load / store

template <class T>
struct SiteIO;

template <>
struct SiteIO<float> {
    static __device__ __forceinline__ void load(const float* X, int64_t nsites, int64_t site,
                                                cpx<float> a[5], cpx<float> b[5]) {
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(X) + m * nsites + site);
            a[m] = {v.x, v.y};
            b[m] = {v.w, -v.z};  // b = -i bt
        }
    }
    static __device__ __forceinline__ void store(float* X, int64_t nsites, int64_t site,
                                                 const cpx<float> a[5], const cpx<float> b[5]) {
#pragma unroll
        for (int m = 0; m < 5; ++m)  // bt = i b
            reinterpret_cast<float4*>(X)[m * nsites + site] = make_float4(a[m].re, a[m].im, -b[m].im, b[m].re);
    }
};

template <>
struct SiteIO<double> {
    static __device__ __forceinline__ void load(const double* X, int64_t nsites, int64_t site,
                                                cpx<double> a[5], cpx<double> b[5]) {
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const double2* p = reinterpret_cast<const double2*>(X) + 2 * (m * nsites + site);
            const double2 va = __ldg(p), vb = __ldg(p + 1);
            a[m] = {va.x, va.y};
            b[m] = {vb.y, -vb.x};
        }
    }
    static __device__ __forceinline__ void store(double* X, int64_t nsites, int64_t site,
                                                 const cpx<double> a[5], const cpx<double> b[5]) {
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            double2* p = reinterpret_cast<double2*>(X) + 2 * (m * nsites + site);
            p[0] = make_double2(a[m].re, a[m].im);
            p[1] = make_double2(-b[m].im, b[m].re);
        }
    }
};

// ------------------------------------------------------------------ kinetic stencil
//
// One axis of the kinetic operator, I'_1 I'_1 I'_2 I'_2 with I'_c = S_c C' S^T_c C (Sec. VII.B;
// the I'_2 blocks act first; S_c moves qubit c one site toward +x: c(j) <- c(j-1)), is linear
// and translation invariant with a dependency cone of +-4 sites.  In the (a, bt) basis its
// coefficients are integers / 16.  They are derived here at compile time by running the four
// blocks on a unit impulse, so the table is the block definition itself, not a transcription.
//
//   K1: C' = C,        C (a,bt) = (1-i)/2 [[1, 1], [-1, 1]] (a, bt)
//   K2: C' = C^dagger, C (a,bt) = (1+i)/2 [[1, -1], [1, 1]] (a, bt),  C^dagger as K1's C
// The scalar prefactors of the eight collides multiply to 1/16 for both variants.

struct KinStencil {
    // g[dst][src][k + 4]: out_dst(j) = 1/16 * sum_k g * in_src(j + k), dst/src 0 = a, 1 = bt
    int g[2][2][9];
};

constexpr void collide_int(int v[2][11], int m00, int m01, int m10, int m11) {
    for (int i = 0; i < 11; ++i) {
        const int a = v[0][i], b = v[1][i];
        v[0][i] = m00 * a + m01 * b;
        v[1][i] = m10 * a + m11 * b;
    }
}

// dir = +1: S_c, c(j) <- c(j-1); dir = -1: S^T_c, c(j) <- c(j+1)
constexpr void shift_int(int v[2][11], int c, int dir) {
    int t[11] = {};
    for (int i = 0; i < 11; ++i) {
        const int src = i - dir;
        t[i] = (src >= 0 && src < 11) ? v[c][src] : 0;
    }
    for (int i = 0; i < 11; ++i) v[c][i] = t[i];
}

constexpr KinStencil make_stencil(int variant) {
    KinStencil S{};
    const int block_qubit[4] = {1, 1, 0, 0};
    for (int src = 0; src < 2; ++src) {
        int v[2][11] = {};
        v[src][5] = 1;  // unit impulse at site 0 (index 5)
        for (int blk = 0; blk < 4; ++blk) {
            const int c = block_qubit[blk];
            if (variant == 0) collide_int(v, 1, 1, -1, 1);
            else collide_int(v, 1, -1, 1, 1);
            shift_int(v, c, -1);
            collide_int(v, 1, 1, -1, 1);
            shift_int(v, c, +1);
        }
        // response at site o feeds out(j) from in(j - o): g[dst][src][k] = v[dst][5 - k]
        for (int dst = 0; dst < 2; ++dst)
            for (int k = -4; k <= 4; ++k) S.g[dst][src][k + 4] = v[dst][5 - k];
    }
    return S;
}

constexpr KinStencil kStencil[2] = {make_stencil(0), make_stencil(1)};

// f(std::integral_constant<int, 0>) .. f(std::integral_constant<int, N - 1>), in order
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// acc + c x for a compile-time integer c: nothing for 0 (fma(0, x, acc) is not folded under IEEE
// rules), an addition or a subtraction for +-1 (the same rounding as the fma)
template <int C, class T>
__device__ __forceinline__ T ktap(T x, T acc) {
    if constexpr (C == 0) return acc;
    else if constexpr (C == 1) return acc + x;
    else if constexpr (C == -1) return acc - x;
    else return fma(T(C), x, acc);
}

// One tap of an (a, bt) stencil on one neighbour, coefficients (AA, AB; BA, BB):
// acc_a += AA a + AB bt and acc_bt += BA a + BB bt, each component as fma(A., a, fma(.B, bt, acc)).
template <int AA, int AB, int BA, int BB, class T>
__device__ __forceinline__ void kin_tap4(const cpx<T>& a, const cpx<T>& bt, cpx<T>& acc_a, cpx<T>& acc_bt) {
    acc_a.re = ktap<AA>(a.re, ktap<AB>(bt.re, acc_a.re));
    acc_a.im = ktap<AA>(a.im, ktap<AB>(bt.im, acc_a.im));
    acc_bt.re = ktap<BA>(a.re, ktap<BB>(bt.re, acc_bt.re));
    acc_bt.im = ktap<BA>(a.im, ktap<BB>(bt.im, acc_bt.im));
}
// Tap K of the kinetic stencil of VARIANT
template <int VARIANT, int K, class T>
__device__ __forceinline__ void kin_tap(const cpx<T>& a, const cpx<T>& bt, cpx<T>& acc_a, cpx<T>& acc_bt) {
    constexpr KinStencil S = kStencil[VARIANT];
    kin_tap4<S.g[0][0][K], S.g[0][1][K], S.g[1][0][K], S.g[1][1][K]>(a, bt, acc_a, acc_bt);
}

// Kinetic operator of one axis at one site from its 9 neighbours along the axis.
// nb[k][m]: (a, b) of level m at offset k - 4.  Returns (a, b) of the output, scaled exactly.
template <class T, int VARIANT>
__device__ __forceinline__ void kinetic_axis_site(const cpx<T> (*nba)[5], const cpx<T> (*nbb)[5],
                                                  cpx<T> oa[5], cpx<T> ob[5]) {
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        cpx<T> acc_a = {T(0), T(0)}, acc_bt = {T(0), T(0)};
        static_for<9>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const cpx<T> bt = {-nbb[k][m].im, nbb[k][m].re};  // bt = i b
            kin_tap<VARIANT, k>(nba[k][m], bt, acc_a, acc_bt);
        });
        const T s = T(0.0625);
        oa[m] = {s * acc_a.re, s * acc_a.im};
        ob[m] = {s * acc_bt.im, -s * acc_bt.re};  // b = -i bt
    }
}

// ------------------------------------------------------------------ potential unitary
//
// U = exp(-i delta V(psi)), psi = a + b, applied to a and to b (Sec. VII.B; V is the right-hand
// side of Eq. eomspin2 written as V(psi) psi):
//     V = g0 rho 1 + g1 (F_x f_x + F_y f_y + F_z f_z) + (g2/5) s s^dagger,
//     F_nu = psi^dagger f_nu psi,  s_m = (-1)^m conj(psi_{-m}).
// Evaluation: V = c 1 + W with c = (g0 + g2/10) rho, the centre of V's spectral bounds, so
// U = e^{-i delta c} exp(-i delta W).  W is tridiagonal (the spin term: f_+ = f_x + i f_y has
// entries 2, 2 sqrt(3/2), 2 sqrt(3/2), 2 above the diagonal) plus the rank-one singlet term, and
// ||delta W|| <= beta = delta (2 |g1| |F| + |g2| rho / 10) (the spin term has eigenvalues
// g1 |F| m, m = -2..2; the singlet term (g2/5) s s^dagger has eigenvalues g2 rho / 5 and 0).  exp(-i delta W) is applied to the
// vectors psi and d = a - b by its Taylor polynomial (Horner form) of the smallest degree K
// with beta^(K+1)/(K+1)! <= tol; then a = U(psi + d)/2, b = U(psi - d)/2.  K is made uniform
// across the warp, so the loop never diverges.
//
// The input may carry an exact power-of-two scale sigma (the unnormalised kinetic output):
// quadratic forms are multiplied by inv_sigma2 = sigma^-2 and the result by 1/sigma.

constexpr int kTaylorMax = 40;
constexpr double kBetaMax = 4.0;  // beyond this the plain Taylor sum loses accuracy: flagged

struct PotParams {
    double g0, g1, g2, delta;
};

// Constants of the potential in the arithmetic type, computed on the host from PotParams.
template <class T>
struct PotConst {
    T cphase;  // delta (g0 + g2/10): e^{-i delta c} with c = (g0 + g2/10) rho
    T dz;      // delta g1: diagonal spin entry per unit F_z m
    T dr;      // delta g2 / 10: diagonal shift of the singlet term per unit rho
    T e0, e1;  // delta g1, delta g1 sqrt(3/2): off-diagonal spin entries per unit F_+
    T R;       // delta g2 / 5: singlet rank-one term
    T b1, b2;  // 2 |g1| delta, |g2| delta / 10: beta = b1 |F| + b2 rho
    PotConst() = default;
    __host__ __device__ explicit PotConst(const PotParams& P) {
        cphase = T(P.delta * (P.g0 + P.g2 / 10.0));
        dz = T(P.delta * P.g1);
        dr = T(P.delta * P.g2 / 10.0);
        e0 = T(P.delta * P.g1);
        e1 = T(P.delta * P.g1 * 1.2247448713915890491);  // sqrt(3/2)
        R = T(P.delta * P.g2 / 5.0);
        b1 = T(2.0 * fabs(P.g1) * P.delta);
        b2 = T(0.1 * fabs(P.g2) * P.delta);
    }
};

// 1/k, k = 0..kTaylorMax+1 (entry 0 unused): Taylor coefficients without divisions.
template <class T>
struct InvTable {
    T v[kTaylorMax + 2];
};
template <class T>
constexpr InvTable<T> make_inv_table() {
    InvTable<T> t{};
    for (int k = 1; k < kTaylorMax + 2; ++k) t.v[k] = T(1.0 / k);
    return t;
}
__constant__ InvTable<float> c_inv_f = make_inv_table<float>();
__constant__ InvTable<double> c_inv_d = make_inv_table<double>();
__device__ __forceinline__ float inv_k(int k, float) { return c_inv_f.v[k]; }
__device__ __forceinline__ double inv_k(int k, double) { return c_inv_d.v[k]; }

template <class T>
struct TaylorTol;
template <>
struct TaylorTol<double> {
    static constexpr double value = 1.1102230246251565e-16;  // 2^-53
};
// FP32: bound on the truncation relative to the site amplitude, per step.  1e-8 sits below the
// FP32 rounding of one step (~1e-7): tightening it to 1e-9 left the FP32-vs-FP64 drift of the 1D
// and 2D workloads unchanged while costing one more Taylor term in the vortex background.
#ifndef QLGA_F32_TAYLOR_TOL
#define QLGA_F32_TAYLOR_TOL 1e-8f
#endif
template <>
struct TaylorTol<float> {
    static constexpr float value = QLGA_F32_TAYLOR_TOL;
};

// e^{-i x} parts.  FP32: for |x| <= 1/2 the Taylor series of sin and cos to x^9 / x^10
// (truncation below 2e-11, under FP32 rounding); otherwise the CUDA library sincosf.
__device__ __forceinline__ void sin_cos(float x, float* s, float* c) {
    if (fabsf(x) <= 0.5f) {
        const float x2 = x * x;
        *s = x * fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 2.7557319e-6f, -1.9841270e-4f), 8.3333333e-3f),
                               -1.6666667e-1f), 1.0f);
        *c = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -2.7557319e-7f, 2.4801587e-5f), -1.3888889e-3f),
                                    4.1666667e-2f), -0.5f), 1.0f);
    } else {
        sincosf(x, s, c);
    }
}
__device__ __forceinline__ void sin_cos(double x, double* s, double* c) { sincos(x, s, c); }

__device__ __forceinline__ int warp_max_int(int v) {
    return static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>(v)));
}

// Smallest K with beta^(K+1)/(K+1)! <= tol.
template <class T>
__device__ __forceinline__ int taylor_degree(T beta, T tol) {
    int K = 0;
    T term = beta;  // beta^(K+1) / (K+1)!
    while (term > tol && K < kTaylorMax) {
        ++K;
        term *= beta * inv_k(K + 1, T(0));
    }
    return K;
}

// The warp-uniform Taylor degree: the smallest K with beta^(K+1)/(K+1)! <= tol for every lane's
// beta (>= 0).  FP32: from the warp's largest beta (positive floats order as their bit patterns),
// so the loop runs on warp-uniform data; FP64 keeps the per-lane degree and its warp maximum.
template <class T>
__device__ __forceinline__ int warp_taylor_degree(T beta, T tol) {
    if constexpr (std::is_same<T, float>::value) {
        const float bmax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(beta) & 0x7fffffffu));
        return taylor_degree(bmax, tol);
    } else {
        return warp_max_int(taylor_degree(beta, tol));
    }
}

// y = (delta W) x, with the per-site coefficients of W
template <class T>
struct WOp {
    T D[5];        // diagonal: delta (g1 F_z m - g2 rho / 10)
    cpx<T> ep[4];  // (i+1, i) entries: delta g1 c_i F_+ ; (i, i+1) = conj
    cpx<T> u[5];   // u_j = (-1)^{m_j} psi_{4-j} = conj(s_j)
    T R;           // delta g2 / 5 (times inv_sigma2)

    __device__ __forceinline__ void apply(const cpx<T> x[5], cpx<T> y[5]) const {
        cpx<T> t0 = cmul(u[0], x[0]), t1 = cmul(u[1], x[1]);
        t0 = cfma(u[2], x[2], t0);
        t1 = cfma(u[3], x[3], t1);
        t0 = cfma(u[4], x[4], t0);
        const cpx<T> t = R * (t0 + t1);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            // D_i x_i + t * conj(u_i)
            const cpx<T> tu = cmulc(u[i], t);
            y[i] = {fma(D[i], x[i].re, tu.re), fma(D[i], x[i].im, tu.im)};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            y[i] = cfmac(ep[i], x[i + 1], y[i]);
            y[i + 1] = cfma(ep[i], x[i], y[i + 1]);
        }
    }
};

// v <- exp(-i delta W) x by the degree-K Taylor polynomial (Horner form; K is warp-uniform)
template <class T>
__device__ __forceinline__ void horner_step(const cpx<T> x[5], const cpx<T> w[5], cpx<T> v[5], T ik) {
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = {fma(ik, w[i].im, x[i].re), fma(-ik, w[i].re, x[i].im)};
}

// vp <- exp(-i delta W) xp (degree K) and vd <- exp(-i delta W) xd (degree Kd <= K).  Both
// Horner recursions run in one loop so their independent matrix-vector products interleave.
template <class T>
__device__ __forceinline__ void taylor_apply2(const WOp<T>& W, const cpx<T> xp[5], cpx<T> vp[5],
                                              const cpx<T> xd[5], cpx<T> vd[5], int K, int Kd) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        vp[i] = xp[i];
        vd[i] = xd[i];
    }
    int k = K;
    for (; k > Kd; --k) {
        cpx<T> w[5];
        W.apply(vp, w);
        horner_step(xp, w, vp, inv_k(k, T(0)));
    }
    for (; k >= 1; --k) {
        cpx<T> wp[5], wd[5];
        W.apply(vp, wp);
        W.apply(vd, wd);
        const T ik = inv_k(k, T(0));
        horner_step(xp, wp, vp, ik);
        horner_step(xd, wd, vd, ik);
    }
}

// The Taylor sums in a frame turned about the spin z axis (used by the fused 2D FP32 kernels and
// by the FP64 kernels outside the interleaved passes).
//
// A rotation about z multiplies level m by e^{i m phi}; it leaves rho, F_z and the singlet
// relation s_m = (-1)^m conj(psi_{-m}) unchanged (the phase is odd in m) and turns F_+ into
// e^{-i phi} F_+.  With e = F_+ / |F_+| and x' = diag(e^2, e, 1, conj(e), conj(e)^2) x (index order
// m = +2..-2), F_+ becomes the real |F_+|, so W's off-diagonal entries are real and each costs two
// multiply-adds instead of four.  The Taylor polynomial commutes with the (unitary, diagonal)
// change of frame, so the result is the same polynomial in W; the frame is undone by folding
// diag(conj(e)^2, conj(e), 1, e, e^2) into the output phase.
//
// Each Horner step v <- x - (i/k) W v is one pass: W / k is formed once per k (shared by the two
// vectors) and x is the start of every output's multiply-add chain, so the step costs no
// operations beyond the matrix-vector product.
template <class T>
struct WFrameK {
    T D[5];    // diagonal of W / k
    T e0, e1;  // off-diagonal entries of W / k: (0,1) = (3,4) = e0, (1,2) = (2,3) = e1 (real)
    T R;       // singlet coefficient of W / k
};

template <class T>
__device__ __forceinline__ void horner_zframe(const cpx<T> x[5], const cpx<T> v[5], cpx<T> o[5], const WFrameK<T>& Wk,
                                              const cpx<T> u[5]) {
    cpx<T> t0 = cmul(u[0], v[0]);  // one accumulation chain (two split chains cost two more additions)
    t0 = cfma(u[1], v[1], t0);
    t0 = cfma(u[2], v[2], t0);
    t0 = cfma(u[3], v[3], t0);
    t0 = cfma(u[4], v[4], t0);
    const cpx<T> t = Wk.R * t0;  // (s^dagger v) times the singlet coefficient
    // y_i = D_i v_i + conj(u_i) t + (off-diagonal neighbours); o = x - i y:
    // o.re = x.re + y.im, o.im = x.im - y.re
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        T re = fma(Wk.D[i], v[i].im, x[i].re);
        T im = fma(-Wk.D[i], v[i].re, x[i].im);
        re = fma(u[i].re, t.im, re);
        re = fma(-u[i].im, t.re, re);
        im = fma(-u[i].re, t.re, im);
        im = fma(-u[i].im, t.im, im);
        if (i > 0) {
            const T c = (i == 1 || i == 4) ? Wk.e0 : Wk.e1;
            re = fma(c, v[i - 1].im, re);
            im = fma(-c, v[i - 1].re, im);
        }
        if (i < 4) {
            const T c = (i == 0 || i == 3) ? Wk.e0 : Wk.e1;
            re = fma(c, v[i + 1].im, re);
            im = fma(-c, v[i + 1].re, im);
        }
        o[i] = {re, im};
    }
}

// Steps k = K .. K - Kin + 1 of the two Horner recursions of potential_tail_zframe (psi and d
// in the frame, both of degree K) in FP32, for the FP64 kernels; the iterate after them goes to
// (vp, vd) in FP64, and the remaining steps k = K - Kin .. 1 run in FP64 on the exact x.  An error
// e in that iterate reaches the result multiplied by (delta W)^k0 / k0! (k0 = K - Kin >= 1 outer
// steps), at most beta^k0 / k0! |e|; potential_site takes k0 with beta^k0 / k0! <= 2^-31, so the
// FP32 rounding of the inner steps (a few 2^-24 of |x|) stays below the FP64 rounding of the step.
// GB300 runs FP32 at 64 times the FP64 rate.
__device__ __forceinline__ void zframe_inner_fp32(const cpx<double> xp[5], const cpx<double> xd[5],
                                                  const cpx<double> u[5], const double D[5], double ep0,
                                                  double ep1, double R, int K, int Kin, cpx<double> vp[5],
                                                  cpx<double> vd[5]) {
    cpx<float> xpf[5], xdf[5], uf[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        xpf[i] = {float(xp[i].re), float(xp[i].im)};
        xdf[i] = {float(xd[i].re), float(xd[i].im)};
        uf[i] = {float(u[i].re), float(u[i].im)};
    }
    float Df[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) Df[i] = float(D[i]);
    const float e0f = float(ep0), e1f = float(ep1), Rf = float(R);
    auto scaledf = [&](int k) {
        const float ik = inv_k(k, 0.f);
        WFrameK<float> Wk;
#pragma unroll
        for (int i = 0; i < 5; ++i) Wk.D[i] = Df[i] * ik;
        Wk.e0 = e0f * ik;
        Wk.e1 = e1f * ik;
        Wk.R = Rf * ik;
        return Wk;
    };
    cpx<float> Ap[5], Ad[5], Bp[5], Bd[5];
    int k = K;
    {
        const WFrameK<float> Wk = scaledf(k);
        horner_zframe(xpf, xpf, Bp, Wk, uf);
        horner_zframe(xdf, xdf, Bd, Wk, uf);
    }
    --k;
    const int kend = K - Kin;  // the last FP32 step is kend + 1
    for (; k >= kend + 2; k -= 2) {  // B -> A -> B
        WFrameK<float> Wk = scaledf(k);
        horner_zframe(xpf, Bp, Ap, Wk, uf);
        horner_zframe(xdf, Bd, Ad, Wk, uf);
        Wk = scaledf(k - 1);
        horner_zframe(xpf, Ap, Bp, Wk, uf);
        horner_zframe(xdf, Ad, Bd, Wk, uf);
    }
    if (k == kend + 1) {
        const WFrameK<float> Wk = scaledf(k);
        horner_zframe(xpf, Bp, Ap, Wk, uf);
        horner_zframe(xdf, Bd, Ad, Wk, uf);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            vp[i] = {double(Ap[i].re), double(Ap[i].im)};
            vd[i] = {double(Ad[i].re), double(Ad[i].im)};
        }
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            vp[i] = {double(Bp[i].re), double(Bp[i].im)};
            vd[i] = {double(Bd[i].re), double(Bd[i].im)};
        }
    }
}

// The end of potential_site in the z frame: the Taylor sums of exp(-i delta W) on psi (degree K) and d
// (degree Kd <= K) in the z frame, then a = U(psi + d)/2, b = U(psi - d)/2.  Fp = F_+ and the
// other inputs as in potential_site.
// FP64: the first Kin steps (k = K .. K - Kin + 1) of the two sums run in FP32 (see
// zframe_inner_fp32); Kin = 0 in FP32.
template <class T>
__device__ __forceinline__ void potential_tail_zframe(cpx<T> a[5], cpx<T> b[5], const cpx<T> psi[5], const cpx<T> d[5],
                                                      cpx<T> Fp, T rho, T Fz, int K, int Kd, const PotConst<T>& C,
                                                      T inv_sigma2, T out_scale, int Kin = 0) {
    const T fp2 = norm2(Fp);
    cpx<T> e = {T(1), T(0)};
    T fpa = T(0);  // |F_+|; below the smallest normal number it is taken as 0 (its terms are far below rounding)
    if (fp2 > std::numeric_limits<T>::min()) {
        const T r = rsqrt(fp2);
        e = r * Fp;
        fpa = fp2 * r;
    }
    const cpx<T> e2 = cmul(e, e);
    cpx<T> xp[5], xd[5];
    xp[0] = cmul(e2, psi[0]);
    xp[1] = cmul(e, psi[1]);
    xp[2] = psi[2];
    xp[3] = cmulc(e, psi[3]);
    xp[4] = cmulc(e2, psi[4]);
    xd[0] = cmul(e2, d[0]);
    xd[1] = cmul(e, d[1]);
    xd[2] = d[2];
    xd[3] = cmulc(e, d[3]);
    xd[4] = cmulc(e2, d[4]);
    cpx<T> u[5];  // u_j = (-1)^{m_j} psi'_{4-j} = conj(s'_j)
    u[0] = xp[4];
    u[1] = {-xp[3].re, -xp[3].im};
    u[2] = xp[2];
    u[3] = {-xp[1].re, -xp[1].im};
    u[4] = xp[0];
    const T g2r = C.dr * rho, gz = C.dz * Fz;
    const T D[5] = {T(2) * gz - g2r, gz - g2r, -g2r, -gz - g2r, T(-2) * gz - g2r};
    const T ep0 = C.e0 * fpa, ep1 = C.e1 * fpa, R = C.R * inv_sigma2;
    auto scaled = [&](int k) {
        const T ik = inv_k(k, T(0));
        WFrameK<T> Wk;
#pragma unroll
        for (int i = 0; i < 5; ++i) Wk.D[i] = D[i] * ik;
        Wk.e0 = ep0 * ik;
        Wk.e1 = ep1 * ik;
        Wk.R = R * ik;
        return Wk;
    };
    auto finish = [&](const cpx<T> (&vp)[5], const cpx<T> (&vd)[5]) {
        T sn, cs;
        sin_cos(C.cphase * rho, &sn, &cs);
        const cpx<T> ph = {cs * out_scale, -sn * out_scale};  // e^{-i delta c} / (2 sigma)
        cpx<T> q[5];  // the output phase with the frame undone
        q[0] = cmulc(e2, ph);
        q[1] = cmulc(e, ph);
        q[2] = ph;
        q[3] = cmul(e, ph);
        q[4] = cmul(e2, ph);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            a[i] = cmul(q[i], vp[i] + vd[i]);
            b[i] = cmul(q[i], vp[i] - vd[i]);
        }
    };
    // The iterates alternate between the register sets A and B, two steps per pass, so that no
    // step copies its result back (the copies of a loop-carried 5-vector are register moves).
    // Steps k = K .. Kd + 1 act on psi alone (d's Horner sum has degree Kd <= K).
    cpx<T> Ap[5], Ad[5], Bp[5], Bd[5];
    int k = K;
    const bool single = K > Kd;
    bool inner_done = false;
    if constexpr (std::is_same<T, double>::value) {
        if (Kin > 0) {  // warp-uniform; FP64 d takes psi's degree (Kd = K)
            zframe_inner_fp32(xp, xd, u, D, ep0, ep1, R, K, Kin, Bp, Bd);
            k = K - Kin;  // the next step; the iterate is in B
            inner_done = true;
        }
    }
    if (!inner_done) {
        if (single) {
            horner_zframe(xp, xp, Ap, scaled(k), u);
            for (--k; k > Kd; --k) {
                horner_zframe(xp, Ap, Bp, scaled(k), u);
#pragma unroll
                for (int i = 0; i < 5; ++i) Ap[i] = Bp[i];
            }
        }
        if (k == 0) {  // Kd = 0 (rare): d keeps its zeroth-order term
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                Bp[i] = single ? Ap[i] : xp[i];
                Bd[i] = xd[i];
            }
        } else {  // first step of both sums: psi from A (or x), d from x
            const WFrameK<T> Wk = scaled(k);
            if (single) horner_zframe(xp, Ap, Bp, Wk, u);
            else horner_zframe(xp, xp, Bp, Wk, u);
            horner_zframe(xd, xd, Bd, Wk, u);
            --k;
        }
    }
    for (; k >= 2; k -= 2) {  // B -> A -> B
        WFrameK<T> Wk = scaled(k);
        horner_zframe(xp, Bp, Ap, Wk, u);
        horner_zframe(xd, Bd, Ad, Wk, u);
        Wk = scaled(k - 1);
        horner_zframe(xp, Ap, Bp, Wk, u);
        horner_zframe(xd, Ad, Bd, Wk, u);
    }
    if (k == 1) {
        const WFrameK<T> Wk = scaled(1);
        horner_zframe(xp, Bp, Ap, Wk, u);
        horner_zframe(xd, Bd, Ad, Wk, u);
        finish(Ap, Ad);
    } else {
        finish(Bp, Bd);
    }
}

// FP64 kernels run the Taylor sums in the z frame too: with the FP64 tolerance the degree is
// higher, and the frame made the fused and two-pass FP64 2D steps 9% faster (the interleaved
// passes keep the plain form: more spills there).
template <class T>
constexpr bool kZframe64 = std::is_same<T, double>::value;

// Apply U to the pair (a, b) of one site in place.  SPLIT_D: pick the degree for d = a - b
// from its size relative to psi (the FP32 interleaved passes, where delta is 1/8 and d's degree
// is often lower: 15% faster there, and the FP32 per-site kernels); otherwise d uses the degree
// of psi (FP64; the fused 2D and the tiled 1D FP32 kernels, where the one warp-uniform loop over
// both vectors beats the saved Taylor terms: 0.80 vs 0.85 ms per 4096^2 step, 2-3% on 1D).  ZFRAME: run the
// Taylor sums in the z frame (potential_tail_zframe).  The frame costs a fixed ~60 operations per
// site and saves ~26 per vector and Taylor term, so it pays where the warp-uniform degree is about
// 3 or more: the FP32 2D vortex states of the fused warp-strip kernels (2.4% faster at 4096^2)
// and the FP64 kernels that call this function outside the interleaved passes (kZframe64), but
// not the lower FP32 degrees of the 1D workloads (5% slower there).
template <class T, bool SPLIT_D, bool ZFRAME = false>
__device__ __forceinline__ void potential_site(cpx<T> a[5], cpx<T> b[5], const PotConst<T>& C,
                                               T inv_sigma2, T out_scale, unsigned* status) {
    cpx<T> psi[5], d[5];
    T n[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        psi[i] = a[i] + b[i];
        d[i] = a[i] - b[i];
        n[i] = norm2(psi[i]);
    }
    const T pn2 = (n[0] + n[1]) + (n[2] + n[3]) + n[4];
    const T rho = pn2 * inv_sigma2;
    const T Fz = (T(2) * (n[0] - n[4]) + (n[1] - n[3])) * inv_sigma2;
    const T r32 = T(1.2247448713915890491);  // sqrt(3/2)
    cpx<T> Fp = cmulc(psi[0], psi[1]);
    Fp = cfmac(psi[3], psi[4], Fp);
    cpx<T> mid = cmulc(psi[1], psi[2]);
    mid = cfmac(psi[2], psi[3], mid);
    Fp = {fma(r32, mid.re, Fp.re), fma(r32, mid.im, Fp.im)};
    Fp = (T(2) * inv_sigma2) * Fp;  // F_+ = psi^dagger f_+ psi
    const T Fabs = sqrt(fma(Fz, Fz, norm2(Fp)));
    const T beta = fma(C.b1, Fabs, C.b2 * rho);
    if (!(beta <= T(kBetaMax))) atomicOr(status, 1u);  // also catches NaN
    const T tol = TaylorTol<T>::value;
    const int K = warp_taylor_degree(beta, tol);
    int Kd = K;
    if (SPLIT_D) {
        T dn2 = T(0);
#pragma unroll
        for (int i = 0; i < 5; ++i) dn2 += norm2(d[i]);
        int k = 0;
        T term = beta;
        while (k < K && term * term * dn2 > tol * tol * pn2) {
            ++k;
            term *= beta * inv_k(k + 1, T(0));
        }
        Kd = warp_max_int(k);
    }
    if constexpr (ZFRAME) {
        int Kin = 0;
        if constexpr (std::is_same<T, double>::value) {
            // the outer FP64 steps k0: the smallest k0 >= 1 with beta^k0 / k0! <= 2^-31 on every
            // lane; the terms of higher order run in FP32 (zframe_inner_fp32)
            const int k0 = warp_max_int(taylor_degree(beta, 4.656612873077393e-10) + 1);
            Kin = K > k0 ? K - k0 : 0;
        }
        potential_tail_zframe<T>(a, b, psi, d, Fp, rho, Fz, K, Kd, C, inv_sigma2, out_scale, Kin);
        return;
    }
    WOp<T> W;
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
    W.R = C.R * inv_sigma2;
    cpx<T> vp[5], vd[5];
    taylor_apply2(W, psi, vp, d, vd, K, Kd);
    T sn, cs;
    sin_cos(C.cphase * rho, &sn, &cs);
    const cpx<T> ph = {cs * out_scale, -sn * out_scale};  // e^{-i delta c} / (2 sigma)
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        a[i] = cmul(ph, vp[i] + vd[i]);
        b[i] = cmul(ph, vp[i] - vd[i]);
    }
}

// ------------------------------------------------------------------ observables
//
// Per-site terms of the boson field psi = a + b, accumulated in FP64 (Sec. III.B Eq. cmap; the
// energy density is the functional whose variation is V(psi) psi, plus the forward-difference
// gradient; the overlap gives the discrete energy of Sec. IV.B).  Order of the accumulators:
enum ObsIndex {
    OBS_NORM_QUBIT = 0,
    OBS_NORM_BOSON = 1,
    OBS_POP0 = 2,  // 2..6: m = +2..-2
    OBS_ENERGY = 7,
    OBS_SINGLET_RE = 8,
    OBS_SINGLET_IM = 9,
    OBS_THETA2 = 10,
    OBS_RHO2 = 11,
    OBS_OVERLAP_RE = 12,
    OBS_OVERLAP_IM = 13,
    OBS_COUNT = 14
};

}  // namespace qlga
