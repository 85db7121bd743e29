// qlga_obs.cuh -- pieces shared by the observable kernels: pair loads in both layouts, the
// per-site spin and singlet terms, and the summation helpers of the deterministic reductions.
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"

namespace qlga {

// Pair load (a, b) of level m at a site from a buffer in the resident layout (a, bt = i b).
template <class T>
__device__ __forceinline__ void load_pair(const T* X, int64_t nsites, int m, int64_t site,
                                          cpx<T>& a, cpx<T>& b);
template <>
__device__ __forceinline__ void load_pair<float>(const float* X, int64_t nsites, int m,
                                                 int64_t site, cpx<float>& a, cpx<float>& b) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(X) + m * nsites + site);
    a = {v.x, v.y};
    b = {v.w, -v.z};  // resident bt = i b
}
template <>
__device__ __forceinline__ void load_pair<double>(const double* X, int64_t nsites, int m,
                                                  int64_t site, cpx<double>& a, cpx<double>& b) {
    const double2* p = reinterpret_cast<const double2*>(X) + 2 * (m * nsites + site);
    const double2 va = __ldg(p), vb = __ldg(p + 1);
    a = {va.x, va.y};
    b = {vb.y, -vb.x};
}

// Pair load from a buffer in the ABI layout (a.re, a.im, b.re, b.im).
template <class T>
__device__ __forceinline__ void load_pair_abi(const T* X, int64_t nsites, int m, int64_t site,
                                              cpx<T>& a, cpx<T>& b) {
    const T* p = X + 4 * (m * nsites + site);
    a = {p[0], p[1]};
    b = {p[2], p[3]};
}

// Local terms of one site from its boson field psi (Sec. III.B): |F|^2, with F_z = psi^dagger f_z
// psi and F_+ = psi^dagger f_+ psi (f_+ = f_x + i f_y, so |F|^2 = F_z^2 + |F_+|^2), and the singlet
// pair amplitude theta = psi^T J psi = 2 psi_2 psi_-2 - 2 psi_1 psi_-1 + psi_0^2.
template <class T>
__device__ __forceinline__ void obs_local(const cpx<T> psi[5], T& F2, cpx<T>& th) {
    const T r32 = T(1.2247448713915890491);  // sqrt(3/2)
    const T Fz = T(2) * (norm2(psi[0]) - norm2(psi[4])) + (norm2(psi[1]) - norm2(psi[3]));
    cpx<T> Fp = cmulc(psi[0], psi[1]) + cmulc(psi[3], psi[4]);
    const cpx<T> mid = cmulc(psi[1], psi[2]) + cmulc(psi[2], psi[3]);
    Fp = {T(2) * (Fp.re + r32 * mid.re), T(2) * (Fp.im + r32 * mid.im)};
    F2 = Fz * Fz + norm2(Fp);
    const cpx<T> t1 = cmul(psi[0], psi[4]), t2 = cmul(psi[1], psi[3]), t3 = cmul(psi[2], psi[2]);
    th = {T(2) * (t1.re - t2.re) + t3.re, T(2) * (t1.im - t2.im) + t3.im};
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-thread accumulator: FP64 for an FP64 state; compensated (Kahan) FP32 for an FP32 state,
// whose per-site terms carry FP32 rounding anyway.  Block and grid sums are FP64.
template <class T>
struct ThreadSum;
template <>
struct ThreadSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct ThreadSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) - double(c); }
};

// Neumaier-compensated running sum.
struct CompSum {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double v) {
        const double t = s + v;
        c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
};

}  // namespace qlga
