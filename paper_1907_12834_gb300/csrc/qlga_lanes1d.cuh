// qlga_lanes1d.cuh -- the fused 1D step with each site spread over five or ten lanes.
//
// On a small 1D lattice one site per thread leaves most of the GPU idle: 1024 sites are 32 warps,
// and in FP64 each warp's Taylor recursions of exp(-i delta W) run on one sub-partition's FP64
// unit.  Here a site's levels m = +2 .. -2 (index 0..4) sit on five lanes (LPS = 5: six sites per
// warp, each lane carrying both recursions, on psi = a + b and on d = a - b) or on ten lanes
// (LPS = 10: three sites per warp; lanes 0..4 of a site carry the psi recursion, lanes 5..9 the d
// recursion, so each lane's chain of dependent work is half as long).  Lanes 30 and 31 repeat
// lanes 0 and 1 of the last site and store nothing.
//   - the kinetic operator K (Sec. VII.B) acts on each level separately: each lane applies the
//     nine-point stencil of its own level to the state held pending K as (P, Q) (qlga_batch1d.cuh),
//     and the lane stores its level of the new held state as (P, Q);
//   - U = e^{-i delta c} exp(-i delta W) needs the site's rho, F_z, F_+ and the singlet vector
//     s_m = (-1)^m conj(psi_{-m}): sums over the site's five psi lanes and shuffles from the lane
//     of level -m;
//   - W is tridiagonal (the spin term) plus the rank-one singlet term, so one application of W to
//     a lane-distributed vector takes each lane's two neighbours and one five-lane sum; the
//     Horner recursion runs with one component per lane.
// The arithmetic is that of potential_site (qlga_device.cuh) component by component; only the
// order of a few sums differs.
#pragma once

#include <cuda_runtime.h>

#include "qlga_batch1d.cuh"  // Pair4, load_raw_pair, store_raw_pair
#include "qlga_device.cuh"

namespace qlga {


template <class T>
__device__ __forceinline__ T lanes_shfl(T v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}
template <class T>
__device__ __forceinline__ cpx<T> lanes_shfl(cpx<T> v, int src) {
    return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

// Sum over the five lanes gb .. gb + 4 of a site, in a fixed order (every lane of the group gets
// the same value).
template <class V>
__device__ __forceinline__ V group5_sum(V v, int gb) {
    const V s0 = lanes_shfl(v, gb), s1 = lanes_shfl(v, gb + 1), s2 = lanes_shfl(v, gb + 2);
    const V s3 = lanes_shfl(v, gb + 3), s4 = lanes_shfl(v, gb + 4);
    return ((s0 + s1) + (s2 + s3)) + s4;
}

// This lane's share of W: y_m = D x_m + conj(u_m) t + conj(ep_m) x_{m+1} + ep_{m-1} x_{m-1}, with
// t = R sum_j u_j x_j (the same entries as WOp).
template <class T>
struct WLane {
    T D;
    cpx<T> up, dn;  // ep_m (0 for m = 4) and ep_{m-1} (0 for m = 0)
    cpx<T> u;
    T R;
    int gb, m;

    __device__ __forceinline__ cpx<T> apply(cpx<T> x) const {
        const cpx<T> xu = lanes_shfl(x, gb + (m < 4 ? m + 1 : 4));
        const cpx<T> xd = lanes_shfl(x, gb + (m > 0 ? m - 1 : 0));
        const cpx<T> t = R * group5_sum(cmul(u, x), gb);
        const cpx<T> tu = cmulc(u, t);
        cpx<T> y = {fma(D, x.re, tu.re), fma(D, x.im, tu.im)};
        y = cfmac(up, xu, y);
        return cfma(dn, xd, y);
    }
};

// One fused step (K, then U with the lattice's constants) of a single periodic 1D lattice of L
// sites, in -> out in the resident layout; 30 / LPS sites per warp, one warp per CTA.
template <class T, int VARIANT, int LPS>
__global__ void __launch_bounds__(32) k_step1d_lanes(const T* __restrict__ in, T* __restrict__ out, int L,
                                                     PotConst<T> C, unsigned* status) {
    static_assert(LPS == 5 || LPS == 10, "five or ten lanes per site");
    constexpr int SPW = 30 / LPS;  // sites per warp
    const int lane = threadIdx.x;
    const int q = lane < 30 ? lane / LPS : SPW - 1;
    const int r = lane < 30 ? lane - LPS * q : lane - 30;
    const int m = r % 5;
    const int chain = LPS == 10 ? r / 5 : 0;  // 1: this lane carries the d recursion alone
    const int gb = LPS * q;                   // the site's psi lanes: gb .. gb + 4
    const int j0 = int(blockIdx.x) * SPW + q;
    const bool store = lane < 30 && chain == 0 && j0 < L;
    const int j = j0 < L ? j0 : L - 1;  // sites past the end redo the last one and store nothing

    // K on level m: the nine-point stencil of the axis (16 times the true value)
    cpx<T> xa = {T(0), T(0)}, xbt = {T(0), T(0)};
    static_for<9>([&](auto kc) {
        constexpr int kk = decltype(kc)::value;
        int jj = j - 4 + kk;
        jj %= L;
        jj = jj < 0 ? jj + L : jj;
        const Pair4<T> p = load_raw_pair(in, int64_t(m) * L + jj);
        kin_tap_pq<VARIANT, kk>(cpx<T>{p.v[0], p.v[1]}, cpx<T>{p.v[2], p.v[3]}, xa, xbt);  // held (P, Q)
    });
    const cpx<T> a = xa, b = {xbt.im, -xbt.re};  // b = -i bt
    const cpx<T> psi = a + b, d = a - b;

    // V(psi) of the site (as potential_site, inputs 16 times the true value: inv_sigma2 = 1/256)
    const T inv_sigma2 = T(1.0 / 256.0), out_scale = T(0.5 / 16.0);
    const T n = norm2(psi);
    const T pn2 = group5_sum(n, gb);
    const T rho = pn2 * inv_sigma2;
    const T Fz = group5_sum(T(2 - m) * n, gb) * inv_sigma2;
    const T r32 = T(1.2247448713915890491);  // sqrt(3/2)
    const cpx<T> psi_up = lanes_shfl(psi, gb + (m < 4 ? m + 1 : 4));
    const cpx<T> fterm = m < 4 ? (m == 0 || m == 3 ? T(1) : r32) * cmulc(psi, psi_up) : cpx<T>{T(0), T(0)};
    const cpx<T> Fp = (T(2) * inv_sigma2) * group5_sum(fterm, gb);  // F_+ = psi^dagger f_+ psi
    const T Fabs = sqrt(fma(Fz, Fz, norm2(Fp)));
    const T beta = fma(C.b1, Fabs, C.b2 * rho);
    if (!(beta <= T(kBetaMax))) atomicOr(status, 1u);  // also catches NaN
    const T tol = TaylorTol<T>::value;
    const int K = warp_max_int(taylor_degree(beta, tol));
    int Kd = K;
    if (sizeof(T) == 4) {  // d's degree from its size relative to psi (as potential_site in FP32)
        const T dn2 = group5_sum(norm2(d), gb);
        int k = 0;
        T term = beta;
        while (k < K && term * term * dn2 > tol * tol * pn2) {
            ++k;
            term *= beta * inv_k(k + 1, T(0));
        }
        Kd = warp_max_int(k);
    }
    WLane<T> W;
    W.gb = gb + 5 * chain;  // the lanes of this lane's recursion
    W.m = m;
    W.D = T(2 - m) * (C.dz * Fz) - C.dr * rho;
    const T e_up = (m == 0 || m == 3) ? C.e0 : C.e1;   // entry (m, m+1) per unit F_+
    const T e_dn = (m == 1 || m == 4) ? C.e0 : C.e1;   // entry (m-1, m)
    W.up = m < 4 ? e_up * Fp : cpx<T>{T(0), T(0)};
    W.dn = m > 0 ? e_dn * Fp : cpx<T>{T(0), T(0)};
    const cpx<T> pm = lanes_shfl(psi, gb + 4 - m);     // psi_{-m}
    W.u = (m & 1) ? cpx<T>{-pm.re, -pm.im} : pm;       // u_m = (-1)^m psi_{-m} = conj(s_m)
    W.R = C.R * inv_sigma2;

    // Horner: v <- x + (-i / k) W v, k = K .. 1 (d from k = Kd).  FP64: the inner steps
    // k = K .. k0 + 1 run in FP32 and the k0 outer ones in FP64 on the exact x, as in
    // zframe_inner_fp32 (beta^k0 / k0! <= 2^-31 on every lane, k0 >= 1), so that the FP32 rounding
    // of the inner iterate reaches the result below the FP64 rounding of the step.
    int k = K;
    [[maybe_unused]] WLane<float> Wf;
    [[maybe_unused]] int k0 = K;
    if constexpr (std::is_same<T, double>::value) {
        k0 = warp_max_int(taylor_degree(beta, 4.656612873077393e-10) + 1);
        k0 = k0 < K ? k0 : K;
        Wf.D = float(W.D);
        Wf.up = {float(W.up.re), float(W.up.im)};
        Wf.dn = {float(W.dn.re), float(W.dn.im)};
        Wf.u = {float(W.u.re), float(W.u.im)};
        Wf.R = float(W.R);
        Wf.gb = W.gb;
        Wf.m = W.m;
    }
    auto to_f = [](cpx<T> z) { return cpx<float>{float(z.re), float(z.im)}; };
    auto to_t = [](cpx<float> z) { return cpx<T>{T(z.re), T(z.im)}; };
    cpx<T> vp, vd;
    if (LPS == 5) {
        vp = psi;
        vd = d;
        if constexpr (std::is_same<T, double>::value) {
            if (K > k0) {  // warp-uniform; FP64 d takes psi's degree (Kd = K)
                const cpx<float> xpf = to_f(psi), xdf = to_f(d);
                cpx<float> vpf = xpf, vdf = xdf;
                for (; k > k0; --k) {
                    const float ik = inv_k(k, 0.f);
                    const cpx<float> wp = Wf.apply(vpf), wd = Wf.apply(vdf);
                    vpf = {fmaf(ik, wp.im, xpf.re), fmaf(-ik, wp.re, xpf.im)};
                    vdf = {fmaf(ik, wd.im, xdf.re), fmaf(-ik, wd.re, xdf.im)};
                }
                vp = to_t(vpf);
                vd = to_t(vdf);
            }
        }
        for (; k >= 1; --k) {
            const T ik = inv_k(k, T(0));
            const cpx<T> wp = W.apply(vp);
            if (k <= Kd) {  // warp-uniform
                const cpx<T> wd = W.apply(vd);
                vd = {fma(ik, wd.im, d.re), fma(-ik, wd.re, d.im)};
            }
            vp = {fma(ik, wp.im, psi.re), fma(-ik, wp.re, psi.im)};
        }
    } else {
        const cpx<T> x = chain == 0 ? psi : d;
        const int kmax = chain == 0 ? K : Kd;
        cpx<T> v = x;
        if constexpr (std::is_same<T, double>::value) {
            if (K > k0) {  // warp-uniform; FP64: kmax = K on both chains
                const cpx<float> xf = to_f(x);
                cpx<float> vf = xf;
                for (; k > k0; --k) {
                    const float ik = inv_k(k, 0.f);
                    const cpx<float> w = Wf.apply(vf);
                    vf = {fmaf(ik, w.im, xf.re), fmaf(-ik, w.re, xf.im)};
                }
                v = to_t(vf);
            }
        }
        for (; k >= 1; --k) {  // every lane applies W (its shuffles take the whole warp)
            const T ik = inv_k(k, T(0));
            const cpx<T> w = W.apply(v);
            if (k <= kmax) v = {fma(ik, w.im, x.re), fma(-ik, w.re, x.im)};
        }
        const cpx<T> other = lanes_shfl(v, gb + 5 * (1 - chain) + m);
        vp = chain == 0 ? v : other;
        vd = chain == 0 ? other : v;
    }
    T sn, cs;
    sin_cos(C.cphase * rho, &sn, &cs);
    const cpx<T> ph = {cs * out_scale, -sn * out_scale};  // e^{-i delta c} / (2 sigma)
    const cpx<T> na = cmul(ph, vp + vd), nb = cmul(ph, vp - vd);
    if (store) store_raw_pq(out, int64_t(m) * L + j, na, nb);  // held pending K again, as (P, Q)
}

}  // namespace qlga
