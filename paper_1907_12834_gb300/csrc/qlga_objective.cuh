// qlga_objective.cuh -- the scalar objectives of a state that gradients are taken of, and their
// cotangents: the population of one level, the singlet fraction and the energy of the boson
// field psi = a + b (Sec. III.B Eq. cmap; the energy functional whose variation is the
// right-hand side of Eq. eomspin2, with forward differences for the gradient term).
//
//   P     = sum |a_l|^2 + |b_l|^2                                   (level l)
//   S     = Theta2 / R2,  Theta2 = sum |psi^T J psi|^2,  R2 = sum rho^2
//   E     = sum_sites [ sum_axis sum_m |psi_m(j+1) - psi_m(j)|^2
//                       + g0/2 rho^2 + g1/2 |F|^2 + g2/10 |psi^T J psi|^2 ]
//
// Cotangents follow the convention gbar = dL/dRe z + i dL/dIm z of a real loss L (so that
// dL = Re sum conj(gbar) dz).  With theta = psi^T J psi, d theta / d psi_k = 2 (-1)^k psi_{-k}, and
// d rho / d conj(psi_k) = psi_k:
//   gbar_psi_k(|theta|^2) = 4 (-1)^k theta conj(psi_{-k}),      gbar_psi_k(rho^2) = 4 rho psi_k,
//   gbar_psi_k(|F|^2)     = 4 (F.f psi)_k,
//   gbar_psi_k(E)         = 2 [ sum_axis (2 psi(j) - psi(j+1) - psi(j-1))
//                               + g0 rho psi + g1 (F.f psi) + (g2/5) (-1)^k theta conj(psi_{-k}) ]_k,
// i.e. twice the discrete kinetic term plus V(psi) psi.  Since psi = a + b, a and b receive the
// same cotangent from S and E; P adds 2 a_l and 2 b_l on level l.
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"
#include "qlga_obs.cuh"

namespace qlga {

constexpr int kObjThreads = 256;
enum ObjIndex { OBJ_POP = 0, OBJ_THETA2 = 1, OBJ_RHO2 = 2, OBJ_ENERGY = 3, OBJ_F2 = 4, OBJ_COUNT = 5 };

// psi = a + b of the 5 levels at a site of an ABI-layout state; the level pairs too when asked.
template <class T>
__device__ __forceinline__ void obj_psi(const T* X, int64_t nsites, int64_t site, cpx<T> psi[5]) {
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        cpx<T> a, b;
        load_pair_abi<T>(X, nsites, m, site, a, b);
        psi[m] = a + b;
    }
}

// Per-block sums (FP64, compensated per thread for FP32 states) of P, Theta2, R2, E and
// sum |F|^2 into partials[block][OBJ_COUNT].
template <class T>
__global__ void __launch_bounds__(kObjThreads) k_objective_sums(const T* __restrict__ X, int64_t nx, int64_t ny,
                                                                int ndim, int level, double g0, double g1,
                                                                double g2, double* __restrict__ partials) {
    const int64_t nsites = nx * ny;
    ThreadSum<T> acc[OBJ_COUNT];
    const T hg0 = T(0.5 * g0), hg1 = T(0.5 * g1), tg2 = T(0.1 * g2);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t site = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; site < nsites; site += stride) {
        const int64_t x = site % nx, y = site / nx;
        cpx<T> psi[5];
        T rho = T(0);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            cpx<T> a, b;
            load_pair_abi<T>(X, nsites, m, site, a, b);
            if (m == level) acc[OBJ_POP].add(norm2(a) + norm2(b));
            psi[m] = a + b;
            rho += norm2(psi[m]);
        }
        T F2;
        cpx<T> th;
        obs_local(psi, F2, th);
        const T th2 = norm2(th);
        T grad = T(0);
        for (int ax = 0; ax < ndim; ++ax) {
            const int64_t xn = ax == 0 ? (x + 1 == nx ? 0 : x + 1) : x;
            const int64_t yn = ax == 1 ? (y + 1 == ny ? 0 : y + 1) : y;
            cpx<T> pn[5];
            obj_psi<T>(X, nsites, yn * nx + xn, pn);
#pragma unroll
            for (int m = 0; m < 5; ++m) grad += norm2(pn[m] - psi[m]);
        }
        acc[OBJ_THETA2].add(th2);
        acc[OBJ_RHO2].add(rho * rho);
        acc[OBJ_ENERGY].add(grad + hg0 * rho * rho + hg1 * F2 + tg2 * th2);
        acc[OBJ_F2].add(F2);
    }
    __shared__ double sh[kObjThreads / 32][OBJ_COUNT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < OBJ_COUNT; ++k) {
        const double v = warp_sum(acc[k].value());
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < OBJ_COUNT) {
        double s = 0.0;
        for (int w = 0; w < kObjThreads / 32; ++w) s += sh[w][threadIdx.x];
        partials[int64_t(blockIdx.x) * OBJ_COUNT + threadIdx.x] = s;
    }
}

// Cotangent of L = w_pop P + w_sing S + w_en E at every site, in the ABI layout.  sums: the
// reduced OBJ_COUNT sums of the same state (device memory).
template <class T>
__global__ void __launch_bounds__(kObjThreads) k_objective_cot(const T* __restrict__ X, T* __restrict__ cot,
                                                               int64_t nx, int64_t ny, int ndim, int level,
                                                               double g0, double g1, double g2,
                                                               const double* __restrict__ sums, double w_pop,
                                                               double w_sing, double w_en) {
    const int64_t nsites = nx * ny;
    const double R2 = sums[OBJ_RHO2], Th2 = sums[OBJ_THETA2];
    // S = Th2 / R2: dS = dTh2 / R2 - Th2 / R2^2 dR2
    const T c_th = R2 > 0.0 ? T(4.0 * w_sing / R2) : T(0);
    const T c_rho = R2 > 0.0 ? T(-4.0 * w_sing * Th2 / (R2 * R2)) : T(0);
    const T e2 = T(2.0 * w_en), e_g0 = T(2.0 * w_en * g0), e_g1 = T(2.0 * w_en * g1), e_g2 = T(0.4 * w_en * g2);
    const T p2 = T(2.0 * w_pop);
    const T c[4] = {T(2), T(2.4494897427831780982), T(2.4494897427831780982), T(2)};  // f_+ entries
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t site = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; site < nsites; site += stride) {
        const int64_t x = site % nx, y = site / nx;
        cpx<T> psi[5];
        obj_psi<T>(X, nsites, site, psi);
        T rho = T(0);
#pragma unroll
        for (int m = 0; m < 5; ++m) rho += norm2(psi[m]);
        T F2;
        cpx<T> th;
        obs_local(psi, F2, th);
        const T Fz = T(2) * (norm2(psi[0]) - norm2(psi[4])) + (norm2(psi[1]) - norm2(psi[3]));
        cpx<T> Fp = {T(0), T(0)};  // F_+ = psi^dagger f_+ psi = sum_i c_i conj(psi_i) psi_{i+1}
#pragma unroll
        for (int i = 0; i < 4; ++i) Fp = cfmac(psi[i], c[i] * psi[i + 1], Fp);
        // discrete kinetic term: sum over axes of 2 psi(j) - psi(j+1) - psi(j-1)
        cpx<T> lap[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) lap[m] = {T(0), T(0)};
        for (int ax = 0; ax < ndim; ++ax) {
            const int64_t xp = ax == 0 ? (x + 1 == nx ? 0 : x + 1) : x, xm = ax == 0 ? (x == 0 ? nx - 1 : x - 1) : x;
            const int64_t yp = ax == 1 ? (y + 1 == ny ? 0 : y + 1) : y, ym = ax == 1 ? (y == 0 ? ny - 1 : y - 1) : y;
            cpx<T> pp[5], pm[5];
            obj_psi<T>(X, nsites, yp * nx + xp, pp);
            obj_psi<T>(X, nsites, ym * nx + xm, pm);
#pragma unroll
            for (int m = 0; m < 5; ++m) lap[m] = lap[m] + (T(2) * psi[m] - pp[m] - pm[m]);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            // (F.f psi)_k = F_z m_k psi_k + (F_+ c_{k-1} psi_{k-1} + conj(F_+) c_k psi_{k+1}) / 2
            cpx<T> Ff = (Fz * T(2 - k)) * psi[k];
            if (k > 0) Ff = Ff + (T(0.5) * c[k - 1]) * cmul(Fp, psi[k - 1]);
            if (k < 4) Ff = Ff + (T(0.5) * c[k]) * cmulc(Fp, psi[k + 1]);
            // (-1)^k theta conj(psi_{-k})
            const T sg = (k & 1) ? T(-1) : T(1);
            const cpx<T> tc = sg * cmul(th, cpx<T>{psi[4 - k].re, -psi[4 - k].im});
            const cpx<T> g = c_th * tc + (c_rho * rho) * psi[k] + e2 * lap[k] + (e_g0 * rho) * psi[k] +
                             e_g1 * Ff + e_g2 * tc;
            cpx<T> a, b;
            load_pair_abi<T>(X, nsites, k, site, a, b);
            cpx<T> ga = g, gb = g;
            if (k == level) {
                ga = ga + p2 * a;
                gb = gb + p2 * b;
            }
            T* p = cot + 4 * (int64_t(k) * nsites + site);
            p[0] = ga.re;
            p[1] = ga.im;
            p[2] = gb.re;
            p[3] = gb.im;
        }
    }
}

}  // namespace qlga
