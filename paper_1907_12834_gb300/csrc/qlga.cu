// qlga.cu -- C ABI and kernels of the GB300 spin-2 QLGA library (arXiv:1907.12834).
//
// The declarations, argument meaning, layout, ownership and error behaviour are in
// include/qlga.h.  This file holds the host side (handle, stream-ordered launches, error
// reporting) and the generic kernels:
//   k_potential      U = exp(-i delta V(psi)) on every site, in place            (Sec. VII.B)
//   k_kinetic_axis   one axis of the kinetic operator, optionally followed by U  (Sec. VII.B)
//   k_observables    FP64 sums of Sec. III.B / IV.B, two-level deterministic reduction
// The fused 2D FP32 step (one HBM read and one write of the state per step) is in
// qlga_step2d.cuh.
//
// Representation.  A plain time step is psi(t+1) = K U(psi(t)) psi(t).  Over n steps this is
// K (U K)^(n-1) U, so the handle keeps the state "pending K": the buffer holds X with the true
// state psi = K X.  Each step is then one fused launch X <- U(K X) K X that reads and writes the
// state once; K is applied on the fly when the true state is read out.  Results are the same
// as applying the operators in the paper's order.
#include "qlga.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "qlga_device.cuh"
#include "qlga_obs.cuh"
#include "qlga_step2d.cuh"
#include "qlga_batch1d.cuh"
#include "qlga_lanes1d.cuh"
#include "qlga_adjoint.cuh"
#include "qlga_interleave.cuh"
#include "qlga_step2d_f64.cuh"
#include "qlga_obs2d.cuh"
#include "qlga_objective.cuh"

#include <vector>

using namespace qlga;

namespace {

constexpr int kThreads = 256;
// Capacity (rows of block partials) of the observables reduction: 8 blocks per SM on a 152-SM
// GB300.  Grids take min(capacity, 8 x the device's SM count) blocks; the loops are grid-stride.
constexpr int kObsMaxBlocks = 1216;
constexpr int64_t kGraphMaxSites = int64_t(1) << 18;  // lattices replayed from step graphs
constexpr int kGraphDefaultSteps = 32;

thread_local std::string g_last_error;

qlga_status fail(qlga_status s, const char* fmt, const char* detail = nullptr) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), fmt, detail ? detail : "");
    g_last_error = buf;
    return s;
}

qlga_status cuda_fail(cudaError_t e, const char* where) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? QLGA_ERR_OOM : QLGA_ERR_CUDA;
}

#define QLGA_CUDA(call, where)                          \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// SM count of the current device, queried once per device (152 on GB300; the fallback only
// applies if the query itself fails, and then the next launch reports the error).
int device_sms() {
    constexpr int kMax = 64;
    static std::atomic<int> cache[kMax];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 152;
    if (dev < kMax) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 152;
    if (dev < kMax) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

// Blocks of the grid-stride observables reduction on the current device.
int obs_blocks_cap() { return std::min(kObsMaxBlocks, 8 * device_sms()); }

}  // namespace

// ===================================================================== kernels

namespace qlga {

// ABI layout <-> resident layout, one (a, b) pair per thread; safe in place.
template <class T, bool TO_RESIDENT>
__global__ void k_convert_layout(const T* src, T* dst, int64_t npairs) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const T a0 = src[4 * i], a1 = src[4 * i + 1], c0 = src[4 * i + 2], c1 = src[4 * i + 3];
        dst[4 * i] = a0;
        dst[4 * i + 1] = a1;
        if (TO_RESIDENT) {  // bt = i b
            dst[4 * i + 2] = -c1;
            dst[4 * i + 3] = c0;
        } else {  // b = -i bt
            dst[4 * i + 2] = c1;
            dst[4 * i + 3] = -c0;
        }
    }
}

// Store a pair (a, b) as (P, Q) = (a + i b, a - i b) at pair index `pair` of the resident layout
// (one float4; the FP64 form is in qlga_step2d_f64.cuh).
__device__ __forceinline__ void put_pq(float* X, int64_t pair, cpx<float> a, cpx<float> b) {
    reinterpret_cast<float4*>(X)[pair] = pq_of(a, b);
}

// U on every site, in place.  All lanes of a warp run the potential (the Taylor degree is a
// warp-wide maximum); lanes past the end work on zeros and store nothing.
// HELD_PQ: store the result as (P, Q) = (a + bt, a - bt), the form in which 1D lattices and the
// fused 2D steps hold a state pending K (qlga_step2d.cuh); else in the resident layout (a, bt).
template <class T, bool SPLIT, bool HELD_PQ = false>
__global__ void __launch_bounds__(kThreads) k_potential(T* X, int64_t nsites, PotConst<T> PC,
                                                        unsigned* status) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < nsites; base += stride) {
        const int64_t site = base + threadIdx.x;
        const bool active = site < nsites;
        cpx<T> a[5], b[5];
        if (active) {
            SiteIO<T>::load(X, nsites, site, a, b);
        } else {
#pragma unroll
            for (int m = 0; m < 5; ++m) a[m] = b[m] = {T(0), T(0)};
        }
        potential_site<T, SPLIT, kZframe64<T>>(a, b, PC, T(1), T(0.5), status);
        if (active) {
            if constexpr (HELD_PQ) {
#pragma unroll
                for (int m = 0; m < 5; ++m) put_pq(X, m * nsites + site, a[m], b[m]);
            } else {
                SiteIO<T>::store(X, nsites, site, a, b);
            }
        }
    }
}

// (a, bt) -> (P, Q) = (a + bt, a - bt) for npairs pairs of the resident layout, in -> out.
template <class T>
__global__ void __launch_bounds__(kThreads) k_pq_of_resident(const T* __restrict__ in, T* __restrict__ out,
                                                             int64_t npairs) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const T* p = in + 4 * i;
        const T ar = p[0], ai = p[1], br = p[2], bi = p[3];
        T* q = out + 4 * i;
        q[0] = ar + br;
        q[1] = ai + bi;
        q[2] = ar - br;
        q[3] = ai - bi;
    }
}

// out = [U o] K_axis(in): the nine-point kinetic stencil of one axis (derived at compile time
// from the block definition), optionally followed by the potential unitary.
template <class T, int VARIANT, bool POT>
__global__ void __launch_bounds__(kThreads) k_kinetic_axis(const T* __restrict__ in,
                                                           T* __restrict__ out, int64_t nx,
                                                           int64_t ny, int axis, PotConst<T> PC,
                                                           unsigned* status) {
    const int64_t nsites = nx * ny;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
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
        cpx<T> oa[5], ob[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            cpx<T> acc_a = {T(0), T(0)}, acc_bt = {T(0), T(0)};
            static_for<9>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                cpx<T> a, b;
                load_pair<T>(in, nsites, m, nb[k], a, b);
                const cpx<T> bt = {-b.im, b.re};  // bt = i b
                kin_tap<VARIANT, k>(a, bt, acc_a, acc_bt);
            });
            const T sc = T(0.0625);
            oa[m] = {sc * acc_a.re, sc * acc_a.im};
            ob[m] = {sc * acc_bt.im, -sc * acc_bt.re};  // b = -i bt
        }
        if (POT) potential_site<T, std::is_same<T, float>::value, kZframe64<T>>(oa, ob, PC, T(1), T(0.5), status);
        if (active) SiteIO<T>::store(out, nsites, site, oa, ob);
    }
}

// a = b = eps psi / 2 from a complex boson field psi5[5][nsites] (re, im interleaved)
template <class T>
__global__ void k_load_boson(const T* __restrict__ psi5, T* __restrict__ X, int64_t nsites, T half_eps) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < 5 * nsites; i += stride) {
        const T re = psi5[2 * i] * half_eps, im = psi5[2 * i + 1] * half_eps;
        X[4 * i + 0] = re;  // a = eps psi / 2
        X[4 * i + 1] = im;
        X[4 * i + 2] = -im;  // bt = i b, b = eps psi / 2
        X[4 * i + 3] = re;
    }
}

// Per-site observable terms in the state's precision, block sums (FP64) into
// partials[block][OBS_COUNT], over the sites [s0, s1) (rows of whole sites: the forward pairs
// wrap periodically only at the lattice's own edge).  X_RESIDENT: X is in the resident layout
// (else the ABI layout); the reference state is always a caller buffer in the ABI layout.
template <class T, bool RESIDENT>
__global__ void __launch_bounds__(kThreads) k_observables(const T* __restrict__ X,
                                                          const T* __restrict__ ref, int64_t nx,
                                                          int64_t ny, int ndim, double g0,
                                                          double g1, double g2,
                                                          double* __restrict__ partials,
                                                          int64_t s0, int64_t s1) {
    const int64_t nsites = nx * ny;
    ThreadSum<T> acc[OBS_COUNT];
    const T hg0 = T(0.5 * g0), hg1 = T(0.5 * g1), tg2 = T(0.1 * g2);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t site = s0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; site < s1; site += stride) {
        const int64_t x = site % nx, y = site / nx;
        cpx<T> psi[5];
        T rho = T(0);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            cpx<T> a, b;
            if (RESIDENT) load_pair<T>(X, nsites, m, site, a, b); else load_pair_abi<T>(X, nsites, m, site, a, b);
            const T pm = norm2(a) + norm2(b);
            acc[OBS_NORM_QUBIT].add(pm);
            acc[OBS_POP0 + m].add(pm);
            psi[m] = a + b;
            rho += norm2(psi[m]);
        }
        acc[OBS_NORM_BOSON].add(rho);
        T F2;
        cpx<T> th;
        obs_local(psi, F2, th);
        const T th2 = norm2(th);
        T grad = T(0);
        for (int ax = 0; ax < ndim; ++ax) {
            const int64_t xn = ax == 0 ? (x + 1 == nx ? 0 : x + 1) : x;
            const int64_t yn = ax == 1 ? (y + 1 == ny ? 0 : y + 1) : y;
            const int64_t sn = yn * nx + xn;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                cpx<T> a, b;
                if (RESIDENT) load_pair<T>(X, nsites, m, sn, a, b); else load_pair_abi<T>(X, nsites, m, sn, a, b);
                grad += norm2((a + b) - psi[m]);
            }
        }
        acc[OBS_ENERGY].add(grad + hg0 * rho * rho + hg1 * F2 + tg2 * th2);
        acc[OBS_SINGLET_RE].add(th.re * T(0.44721359549995793928));  // 1/sqrt(5)
        acc[OBS_SINGLET_IM].add(th.im * T(0.44721359549995793928));
        acc[OBS_THETA2].add(th2);
        acc[OBS_RHO2].add(rho * rho);
        if (ref) {
            cpx<T> ov = {T(0), T(0)};
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                cpx<T> a, b;
                load_pair_abi<T>(ref, nsites, m, site, a, b);  // reference states are caller buffers (ABI layout)
                ov = cfmac(psi[m], a + b, ov);
            }
            acc[OBS_OVERLAP_RE].add(ov.re);
            acc[OBS_OVERLAP_IM].add(ov.im);
        }
    }
    __shared__ double sh[kThreads / 32][OBS_COUNT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < OBS_COUNT; ++k) {
        const double v = warp_sum(acc[k].value());
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < OBS_COUNT) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w][threadIdx.x];
        partials[int64_t(blockIdx.x) * OBS_COUNT + threadIdx.x] = s;
    }
}

// Per-run observables of a batch: one CTA per run; terms in the state's precision (compensated
// per-thread sums for FP32), FP64 block sums in a fixed order; out[run][OBS_COUNT].
template <class T>
__global__ void __launch_bounds__(kThreads) k_batch_observables(const T* __restrict__ X,
                                                                const BatchRun* __restrict__ runs,
                                                                const double* __restrict__ g3,
                                                                double* __restrict__ out) {
    const BatchRun run = runs[blockIdx.x];
    const int L = run.L;
    const int ny = run.ny, nx = L / ny;
    const T hg0 = T(0.5 * g3[3 * blockIdx.x]), hg1 = T(0.5 * g3[3 * blockIdx.x + 1]);
    const T tg2 = T(0.1 * g3[3 * blockIdx.x + 2]);
    ThreadSum<T> acc[OBS_COUNT];
    auto boson = [&](int m, int j) {
        const Pair4<T> p = load_raw_pair(X, run.base + int64_t(m) * L + j);
        return cpx<T>{p.v[0] + p.v[3], p.v[1] - p.v[2]};  // a + b, b = -i bt
    };
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        cpx<T> psi[5];
        T rho = T(0);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const Pair4<T> p = load_raw_pair(X, run.base + int64_t(m) * L + j);
            const T pm = p.v[0] * p.v[0] + p.v[1] * p.v[1] + p.v[2] * p.v[2] + p.v[3] * p.v[3];
            acc[OBS_NORM_QUBIT].add(pm);
            acc[OBS_POP0 + m].add(pm);
            psi[m] = {p.v[0] + p.v[3], p.v[1] - p.v[2]};
            rho += norm2(psi[m]);
        }
        acc[OBS_NORM_BOSON].add(rho);
        T F2;
        cpx<T> th;
        obs_local(psi, F2, th);
        const T th2 = norm2(th);
        // forward differences along x (and y for a 2D run), periodic within the run
        const int x = j % nx, y = j / nx;
        const int jx = y * nx + (x + 1 == nx ? 0 : x + 1);
        T grad = T(0);
#pragma unroll
        for (int m = 0; m < 5; ++m) grad += norm2(boson(m, jx) - psi[m]);
        if (ny > 1) {
            const int jy = (y + 1 == ny ? 0 : y + 1) * nx + x;
#pragma unroll
            for (int m = 0; m < 5; ++m) grad += norm2(boson(m, jy) - psi[m]);
        }
        acc[OBS_ENERGY].add(grad + hg0 * rho * rho + hg1 * F2 + tg2 * th2);
        acc[OBS_SINGLET_RE].add(th.re * T(0.44721359549995793928));
        acc[OBS_SINGLET_IM].add(th.im * T(0.44721359549995793928));
        acc[OBS_THETA2].add(th2);
        acc[OBS_RHO2].add(rho * rho);
    }
    __shared__ double sh[kThreads / 32][OBS_COUNT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < OBS_COUNT; ++k) {
        const double v = warp_sum(acc[k].value());
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < OBS_COUNT) {
        CompSum cs;
        for (int w = 0; w < kThreads / 32; ++w) cs.add(sh[w][threadIdx.x]);
        out[int64_t(blockIdx.x) * OBS_COUNT + threadIdx.x] = cs.s + cs.c;
    }
}

// Per-site fields (see qlga_fields in qlga.h): 11 planes of T.
__device__ __forceinline__ double wrap_pi(double d) {
    const double pi = 3.14159265358979323846;
    return d > pi ? d - 2.0 * pi : (d <= -pi ? d + 2.0 * pi : d);
}

// One site per thread; qlga_fields takes it for 1D lattices (2D lattices: k_fields2d below).
template <class T>
__global__ void __launch_bounds__(kThreads) k_fields(const T* __restrict__ X, T* __restrict__ out,
                                                     int64_t nx, int64_t ny, int ndim) {
    const int64_t nsites = nx * ny;
    const T r32 = T(1.2247448713915890491);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t site = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; site < nsites; site += stride) {
        const int64_t x = site % nx, y = site / nx;
        cpx<T> psi[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            cpx<T> a, b;
            load_pair<T>(X, nsites, m, site, a, b);
            psi[m] = a + b;
        }
        const T Fz = T(2) * (norm2(psi[0]) - norm2(psi[4])) + (norm2(psi[1]) - norm2(psi[3]));
        cpx<T> Fp = cmulc(psi[0], psi[1]) + cmulc(psi[3], psi[4]);
        const cpx<T> mid = cmulc(psi[1], psi[2]) + cmulc(psi[2], psi[3]);
        Fp = {T(2) * (Fp.re + r32 * mid.re), T(2) * (Fp.im + r32 * mid.im)};
        const T fperp = sqrt(norm2(Fp));
        const cpx<T> t1 = cmul(psi[0], psi[4]), t2 = cmul(psi[1], psi[3]), t3 = cmul(psi[2], psi[2]);
        const cpx<T> th = {T(2) * (t1.re - t2.re) + t3.re, T(2) * (t1.im - t2.im) + t3.im};
        const T a00 = sqrt(norm2(th)) * T(0.44721359549995793928);
        const T nrm = sqrt(Fz * Fz + fperp * fperp + a00 * a00);
        out[0 * nsites + site] = Fz;
        out[1 * nsites + site] = fperp;
        out[2 * nsites + site] = a00;
        out[3 * nsites + site] = nrm > T(0) ? fabs(Fz) / nrm : T(0);
        out[4 * nsites + site] = nrm > T(0) ? fperp / nrm : T(0);
        out[5 * nsites + site] = nrm > T(0) ? a00 / nrm : T(0);
        const int64_t xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
        const int64_t yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            double w = 0.0;
            if (ndim == 2) {
                double S[4];  // phases at (x+1,y+1), (x+1,y-1), (x-1,y+1), (x-1,y-1)
                const int64_t nb[4] = {yp * nx + xp, ym * nx + xp, yp * nx + xm, ym * nx + xm};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    cpx<T> a, b;
                    load_pair<T>(X, nsites, m, nb[k], a, b);
                    S[k] = atan2(double(a.im) + double(b.im), double(a.re) + double(b.re));
                }
                const double vy_xp = wrap_pi(S[0] - S[1]) * 0.5, vy_xm = wrap_pi(S[2] - S[3]) * 0.5;
                const double vx_yp = wrap_pi(S[0] - S[2]) * 0.5, vx_ym = wrap_pi(S[1] - S[3]) * 0.5;
                w = (vy_xp - vy_xm - vx_yp + vx_ym) * 0.5;
            }
            out[(6 + m) * nsites + site] = T(w);
        }
    }
}


// The same fields on a 2D lattice, by tiles of kFieldsTx x kFieldsTy sites: the phases of the
// tile and its one-site periodic halo are computed once into shared memory (each site's phase
// serves the four sites whose diagonal neighbour it is: 1.3 phases per site and level instead of
// 4), with the FP32 atan2 of psi = a + b formed in FP64 and rounded once (within a few 1e-7 rad;
// the FP64 atan2 costs 60 times more on GB300).  Each thread reads its own site once: its phases
// fill the tile's interior and its local fields are written before the block's barrier; the first
// kFieldsRing threads read the ring of halo sites.  The kernel waits mostly on its loads, so it
// runs five blocks per SM (48 registers, a few bytes spilled) rather than the four that the 60
// registers the compiler picks alone allow; consecutive tiles fill alternate phase buffers, so one
// barrier per tile suffices.  The four phase differences of the vorticity
// cancel but for their wraps, so it is pi/2 times an integer, the sum of the wrap counts; a count
// is the one place where the phase error could change a result, and a site and level where one of
// its four differences lies within 1e-4 of +-pi takes its four phases again in FP64, so every
// count is the FP64 one and the vorticity is (pi/2) N exactly in either precision.
constexpr int kFieldsTx = 32, kFieldsTy = 8;
constexpr int kFieldsRing = 2 * (kFieldsTx + 2) + 2 * kFieldsTy;  // halo sites around a tile: 84
static_assert(kFieldsRing <= kFieldsTx * kFieldsTy, "one ring site per thread at most");
template <class T>
__global__ void __launch_bounds__(kFieldsTx * kFieldsTy, 5) k_fields2d(const T* __restrict__ X, T* __restrict__ out,
                                                                    int64_t nx, int64_t ny) {
    __shared__ float phb[2][5][kFieldsTy + 2][kFieldsTx + 2];
    int parity = 0;
    const int64_t nsites = nx * ny;
    const T r32 = T(1.2247448713915890491);
    const int64_t tiles_x = (nx + kFieldsTx - 1) / kFieldsTx, tiles_y = (ny + kFieldsTy - 1) / kFieldsTy;
    const int tx = threadIdx.x % kFieldsTx, ty = threadIdx.x / kFieldsTx;
    // the ring entry (hy, hx) of this thread's halo site, for threads below kFieldsRing: the top
    // and bottom rows of the halo box, then its left and right columns
    const int r = threadIdx.x;
    const int ring_hy = r < kFieldsTx + 2 ? 0
                        : r < 2 * (kFieldsTx + 2) ? kFieldsTy + 1
                        : 1 + (r - 2 * (kFieldsTx + 2)) % kFieldsTy;
    const int ring_hx = r < kFieldsTx + 2 ? r
                        : r < 2 * (kFieldsTx + 2) ? r - (kFieldsTx + 2)
                        : (r < 2 * (kFieldsTx + 2) + kFieldsTy ? 0 : kFieldsTx + 1);
    for (int64_t tile = blockIdx.x; tile < tiles_x * tiles_y; tile += gridDim.x) {
        float (*ph)[kFieldsTy + 2][kFieldsTx + 2] = phb[parity];
        const int64_t x0 = (tile % tiles_x) * kFieldsTx, y0 = (tile / tiles_x) * kFieldsTy;
        const int64_t x = x0 + tx, y = y0 + ty;
        const bool inside = x < nx && y < ny;
        {
            // this thread's site, or its periodic image where the tile passes the lattice's edge
            const int64_t site = (y % ny) * nx + (x % nx);
            cpx<T> psi[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                cpx<T> a, b;
                load_pair<T>(X, nsites, m, site, a, b);
                psi[m] = a + b;
                const double re = double(a.re) + double(b.re), im = double(a.im) + double(b.im);
                ph[m][ty + 1][tx + 1] = atan2f(float(im), float(re));
            }
            if (inside) {
                const T Fz = T(2) * (norm2(psi[0]) - norm2(psi[4])) + (norm2(psi[1]) - norm2(psi[3]));
                cpx<T> Fp = cmulc(psi[0], psi[1]) + cmulc(psi[3], psi[4]);
                const cpx<T> mid = cmulc(psi[1], psi[2]) + cmulc(psi[2], psi[3]);
                Fp = {T(2) * (Fp.re + r32 * mid.re), T(2) * (Fp.im + r32 * mid.im)};
                const T fperp = sqrt(norm2(Fp));
                const cpx<T> t1 = cmul(psi[0], psi[4]), t2 = cmul(psi[1], psi[3]), t3 = cmul(psi[2], psi[2]);
                const cpx<T> th = {T(2) * (t1.re - t2.re) + t3.re, T(2) * (t1.im - t2.im) + t3.im};
                const T a00 = sqrt(norm2(th)) * T(0.44721359549995793928);
                const T nrm = sqrt(Fz * Fz + fperp * fperp + a00 * a00);
                out[0 * nsites + site] = Fz;
                out[1 * nsites + site] = fperp;
                out[2 * nsites + site] = a00;
                out[3 * nsites + site] = nrm > T(0) ? fabs(Fz) / nrm : T(0);
                out[4 * nsites + site] = nrm > T(0) ? fperp / nrm : T(0);
                out[5 * nsites + site] = nrm > T(0) ? a00 / nrm : T(0);
            }
        }
        if (r < kFieldsRing) {
            int64_t xx = (x0 - 1 + ring_hx) % nx, yy = (y0 - 1 + ring_hy) % ny;
            xx = xx < 0 ? xx + nx : xx;
            yy = yy < 0 ? yy + ny : yy;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                cpx<T> a, b;
                load_pair<T>(X, nsites, m, yy * nx + xx, a, b);
                const double re = double(a.re) + double(b.re), im = double(a.im) + double(b.im);
                ph[m][ring_hy][ring_hx] = atan2f(float(im), float(re));
            }
        }
        __syncthreads();
        if (inside) {
            const int64_t site = y * nx + x;
            const int64_t xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
            const int64_t yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                // phases at (x+1,y+1), (x+1,y-1), (x-1,y+1), (x-1,y-1): halo index = tile index + 1
                // the four differences cancel but for their wraps, so the vorticity is
                // (pi/2)(n01 - n23 - n02 + n13) with n the wrap count of each difference
                auto count = [](auto d, auto pi) { return d > pi ? -1 : (d <= -pi ? 1 : 0); };
                const float pf = 3.14159265f;
                const float S0 = ph[m][ty + 2][tx + 2], S1 = ph[m][ty][tx + 2];
                const float S2 = ph[m][ty + 2][tx], S3 = ph[m][ty][tx];
                const float d01 = S0 - S1, d23 = S2 - S3, d02 = S0 - S2, d13 = S1 - S3;
                auto near = [&](float d) { return fabsf(fabsf(d) - pf) < 1e-4f; };
                int N = count(d01, pf) - count(d23, pf) - count(d02, pf) + count(d13, pf);
                if (near(d01) || near(d23) || near(d02) || near(d13)) {
                    const int64_t nb[4] = {yp * nx + xp, ym * nx + xp, yp * nx + xm, ym * nx + xm};
                    double S[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        cpx<T> a, b;
                        load_pair<T>(X, nsites, m, nb[k], a, b);
                        S[k] = atan2(double(a.im) + double(b.im), double(a.re) + double(b.re));
                    }
                    const double pd = 3.14159265358979323846;
                    N = count(S[0] - S[1], pd) - count(S[2] - S[3], pd) - count(S[0] - S[2], pd) +
                        count(S[1] - S[3], pd);
                }
                if constexpr (std::is_same<T, float>::value) out[(6 + m) * nsites + site] = 1.57079633f * float(N);
                else out[(6 + m) * nsites + site] = 1.5707963267948966 * double(N);
            }
        }
        parity ^= 1;  // the next tile fills the other buffer: one barrier per tile
    }
}

// out[k] = compensated sum of partials[b][k] over rows b (rows of ncols), in a fixed order: block
// k reduces quantity k, thread t takes rows t, t + 128, ...; each warp's 32 (sum, compensation)
// pairs combine in a fixed butterfly, then thread 0 adds the four warps in order.  Launch with
// ncols blocks of kReduceThreads threads: the FP64 additions of the columns run on ncols SMs.
constexpr int kReduceThreads = 128;
__global__ void __launch_bounds__(kReduceThreads) k_reduce_partials(const double* __restrict__ partials,
                                                                    int nblocks, int ncols,
                                                                    double* __restrict__ out) {
    const int k = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (k >= ncols) return;  // whole block
    CompSum cs;
    for (int b = threadIdx.x; b < nblocks; b += kReduceThreads) cs.add(partials[int64_t(b) * ncols + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, cs.s, o);
        const double oc = __shfl_xor_sync(0xffffffffu, cs.c, o);
        // both lanes of a pair compute the same combination (lower lane's terms first)
        CompSum m;
        if (lane & o) {
            m.add(os);
            m.add(cs.s);
        } else {
            m.add(cs.s);
            m.add(os);
        }
        m.c += (lane & o) ? (oc + cs.c) : (cs.c + oc);
        cs = m;
    }
    __shared__ double ws[kReduceThreads / 32], wc[kReduceThreads / 32];
    if (lane == 0) {
        ws[w] = cs.s;
        wc[w] = cs.c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        CompSum t;
        double c = 0.0;
        for (int i = 0; i < kReduceThreads / 32; ++i) {
            t.add(ws[i]);
            c += wc[i];
        }
        out[k] = t.s + (t.c + c);
    }
}

}  // namespace qlga

// ===================================================================== fused 2D step: launch

namespace qlga {

inline bool step2d_f32_supported(int64_t nx, int64_t ny) {
    return nx % kStep2dWarpCols == 0 && nx >= kStep2dWarpCols && ny >= 1 && nx <= (int64_t(1) << 30) &&
           ny <= (int64_t(1) << 30);
}

// Relative throughput of an SM sub-partition that holds k warps of a fused strip kernel.  FP32:
// the FMA pipe needs about three warps to stay busy (fitted to the 2D step timed at 256^2 ..
// 1024^2 with one, two and three warps per sub-partition: 0.67, 0.90, 1); FP64: one warp keeps
// the FP64 pipe busy (a warp's FP64 FMA holds it for many cycles).
inline double step2d_pipe_eff(bool fp32, int64_t k) {
    if (!fp32 || k >= 3) return 1.0;
    return k == 2 ? 0.90 : 0.67;
}

// Row chunks per strip.  A chunk of r rows costs about r + w row updates: its first 8 rows only
// fill the y pipeline and run the kinetic part of a row update, w = 8 x that part (warm10 = 10 w:
// 32 in FP32, where the kinetic part is ~0.4 of a row update; 18 in FP64, where it is ~0.23).
// With W = strips x chunks warps (at most the resident capacity sms x per_sm) the busiest of the
// 4 sms sub-partitions holds k = ceil(W / (4 sms)) warps and finishes after about
// k / eff(k) x (ceil(ny / chunks) + w) row times.  Within one k more chunks are shorter, so the
// candidates are the largest chunk count of each k; the cheapest is used (the larger on ties).
inline int step2d_chunks(int64_t strips, int64_t ny, int sms, int per_sm, bool fp32, int warm10) {
    int64_t cmax = (int64_t(sms) * per_sm) / strips;
    if (cmax > ny) cmax = ny;
    if (cmax <= 1) return 1;
    const int64_t lanes = 4 * int64_t(sms);
    int64_t best = 1;
    double best_cost = -1.0;
    for (int64_t k = 1;; ++k) {
        int64_t c = (k * lanes) / strips;
        if (c > cmax) c = cmax;
        if (c >= 1) {
            const int64_t kk = (strips * c + lanes - 1) / lanes;
            const double cost = double(kk) / step2d_pipe_eff(fp32, kk) * (double((ny + c - 1) / c) + 0.1 * warm10);
            if (best_cost < 0.0 || cost <= best_cost) {
                best = c;
                best_cost = cost;
            }
        }
        if (c >= cmax) break;
    }
    return int(best);
}

// Per-device launch facts (SM count, resident warp strips per SM), set up once per device.  The
// shared-memory opt-in is a per-device function attribute, so it is applied on each device.
struct Step2dDevice {
    int sms = 0, per_sm = 0, per_sm64 = 0, per_sm_obs = 0;
};

inline int step2d_device(Step2dDevice* out) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static Step2dDevice cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    std::lock_guard<std::mutex> lock(mu);
    Step2dDevice& d = cache[dev];
    if (d.sms == 0) {
        int sms = 0, ctas = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
        const int smem = kStep2dWarpSmemBytes;
        if (cudaFuncSetAttribute(k_step2d_f32<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_step2d_f32<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_step2d_f32<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_step2d_f32<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_batch_step2d_f32<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_batch_step2d_f32<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_batch_step2d_f32<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_batch_step2d_f32<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_step2d_f32<0, true>, kStep2dWarpsPerCta * 32, smem) != cudaSuccess)
            return 1;
        d.per_sm = ctas > 0 ? ctas * kStep2dWarpsPerCta : 1;
        const int s64 = kStep2d64SmemBytes;
        if (cudaFuncSetAttribute(k_step2d_f64<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_step2d_f64<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_step2d_f64<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_step2d_f64<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64) != cudaSuccess) return 1;
        int ctas64 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas64, k_step2d_f64<0, true>, kStep2d64WarpsPerCta * 32, s64) != cudaSuccess)
            return 1;
        d.per_sm64 = ctas64 > 0 ? ctas64 * kStep2d64WarpsPerCta : 1;
        if (cudaFuncSetAttribute(k_obs2d_f32<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_obs2d_f32<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_obs2d_f32<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        if (cudaFuncSetAttribute(k_obs2d_f32<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        int ctas_obs = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_obs, k_obs2d_f32<0, true>, kStep2dWarpsPerCta * 32, smem) != cudaSuccess)
            return 1;
        d.per_sm_obs = ctas_obs > 0 ? ctas_obs * kStep2dWarpsPerCta : 1;
        d.sms = sms;
    }
    *out = d;
    return 0;
}

// FP64: whether the fused kernel beats the two-pass form (x pass, then y pass + U) on an nx x ny
// lattice (nx a multiple of 32).  The fused kernel costs the row-chunk estimate above; the
// two-pass form has no warm-up rows but evaluates the y axis as a second nine-point stencil and
// reads and writes the state twice: 1.135 fused row updates per row of a strip, spread over all
// sub-partitions (calibrated on 4096^2, 56.0 vs 52.4 ms per step).  Short chunks on small lattices
// favour the two-pass form (512^2: 0.93 vs 0.99 ms per step; 384 x 107: 0.21 vs 0.35 ms).
inline bool step2d_f64_fused_preferred(int64_t nx, int64_t ny) {
    Step2dDevice dv;
    if (step2d_device(&dv)) return true;  // the launch reports the error
    const int64_t strips = nx / kStep2dWarpCols;
    const int64_t c = step2d_chunks(strips, ny, dv.sms, dv.per_sm64, false, 18);
    const int64_t lanes = 4 * int64_t(dv.sms);
    const double fused = double((strips * c + lanes - 1) / lanes) * (double((ny + c - 1) / c) + 1.8);
    const double two_pass = 1.135 * double(strips * ny) / double(lanes);
    return fused <= two_pass;
}

// FP64 form (qlga_step2d_f64.cuh); same contract as step2d_f32_launch.
inline int step2d_f64_launch(const double* in, double* out, int64_t nx, int64_t ny, int variant, bool pot,
                             PotConst<double> PC, unsigned* status, cudaStream_t stream) {
    Step2dDevice dv;
    if (step2d_device(&dv)) return 1;
    const int64_t strips = nx / kStep2dWarpCols;
    const int chunks = step2d_chunks(strips, ny, dv.sms, dv.per_sm64, false, 18);
    const int grid = int((strips * chunks + kStep2d64WarpsPerCta - 1) / kStep2d64WarpsPerCta);
    const dim3 b(kStep2d64WarpsPerCta * 32);
    const int smem = kStep2d64SmemBytes;
    if (variant == 0) {
        if (pot) k_step2d_f64<0, true><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
        else k_step2d_f64<0, false><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
    } else {
        if (pot) k_step2d_f64<1, true><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
        else k_step2d_f64<1, false><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
    }
    return cudaPeekAtLastError() != cudaSuccess;
}

// Returns 0 on success (errors are left in cudaGetLastError()).  pot = false applies the kinetic
// operator alone.
inline int step2d_f32_launch(const float* in, float* out, int64_t nx, int64_t ny, int variant, bool pot,
                             PotConst<float> PC, unsigned* status, cudaStream_t stream) {
    Step2dDevice dv;
    if (step2d_device(&dv)) return 1;
    const int64_t strips = nx / kStep2dWarpCols;
    const int chunks = step2d_chunks(strips, ny, dv.sms, dv.per_sm, true, 32);
    const int grid = int((strips * chunks + kStep2dWarpsPerCta - 1) / kStep2dWarpsPerCta);
    const dim3 b(kStep2dWarpsPerCta * 32);
    const int smem = kStep2dWarpSmemBytes;
    if (variant == 0) {
        if (pot) k_step2d_f32<0, true><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
        else k_step2d_f32<0, false><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
    } else {
        if (pot) k_step2d_f32<1, true><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
        else k_step2d_f32<1, false><<<grid, b, smem, stream>>>(in, out, int(nx), int(ny), chunks, PC, status);
    }
    return cudaPeekAtLastError() != cudaSuccess;
}

// Fused observables of a 2D FP32 lattice held pending K (qlga_obs2d.cuh).  Scratch holds the
// two edge buffers (float2 [strips][ny][5] each) and the partial rows; obs2d_scratch_bytes is its
// size (at most ~6 bytes per site beside the 80-byte state).
inline int obs2d_edge_blocks(int64_t strips, int64_t ny) {
    const int64_t b = (strips * ny + kObs2dEdgeThreads - 1) / kObs2dEdgeThreads;
    const int64_t cap = std::min<int64_t>(kObs2dEdgeBlocksMax, 4 * int64_t(device_sms()));
    return int(b < 1 ? 1 : (b > cap ? cap : b));
}

inline size_t obs2d_edge_bytes(int64_t nx, int64_t ny) {
    return (size_t(nx / kStep2dWarpCols) * size_t(ny) * 5 * sizeof(float2) + 255) & ~size_t(255);
}

inline size_t obs2d_scratch_bytes(int64_t nx, int64_t ny, int warps) {
    return 2 * obs2d_edge_bytes(nx, ny) +
           sizeof(double) * OBS_COUNT * size_t(warps + obs2d_edge_blocks(nx / kStep2dWarpCols, ny));
}

// Launches the read-out; on return partials (inside scratch) holds *rows rows of OBS_COUNT sums.
// Returns 0 on success, 1 on a launch error (left in cudaGetLastError()), 2 if scratch is too small.
inline int obs2d_f32_launch(const float* in, const float* ref, int64_t nx, int64_t ny, int variant, double g0,
                            double g1, double g2, void* scratch, size_t scratch_bytes, cudaStream_t stream,
                            double** partials, int* rows) {
    Step2dDevice dv;
    if (step2d_device(&dv)) return 1;
    const int64_t strips = nx / kStep2dWarpCols;
    const int chunks = step2d_chunks(strips, ny, dv.sms, dv.per_sm_obs, true, 32);
    const int warps = int(strips * chunks);
    if (obs2d_scratch_bytes(nx, ny, warps) > scratch_bytes) return 2;
    char* p = static_cast<char*>(scratch);
    float2* edge_l = reinterpret_cast<float2*>(p);
    float2* edge_r = reinterpret_cast<float2*>(p + obs2d_edge_bytes(nx, ny));
    double* part = reinterpret_cast<double*>(p + 2 * obs2d_edge_bytes(nx, ny));
    const int grid = (warps + kStep2dWarpsPerCta - 1) / kStep2dWarpsPerCta;
    const float hg0 = float(0.5 * g0), hg1 = float(0.5 * g1), tg2 = float(0.1 * g2);
    const dim3 b(kStep2dWarpsPerCta * 32);
    const int sm = kStep2dWarpSmemBytes;
    if (variant == 0) {
        if (ref) k_obs2d_f32<0, true><<<grid, b, sm, stream>>>(in, ref, int(nx), int(ny), chunks, hg0, hg1, tg2, edge_l, edge_r, part);
        else k_obs2d_f32<0, false><<<grid, b, sm, stream>>>(in, ref, int(nx), int(ny), chunks, hg0, hg1, tg2, edge_l, edge_r, part);
    } else {
        if (ref) k_obs2d_f32<1, true><<<grid, b, sm, stream>>>(in, ref, int(nx), int(ny), chunks, hg0, hg1, tg2, edge_l, edge_r, part);
        else k_obs2d_f32<1, false><<<grid, b, sm, stream>>>(in, ref, int(nx), int(ny), chunks, hg0, hg1, tg2, edge_l, edge_r, part);
    }
    if (cudaPeekAtLastError() != cudaSuccess) return 1;
    const int eb = obs2d_edge_blocks(strips, ny);
    k_obs2d_edges<<<eb, kObs2dEdgeThreads, 0, stream>>>(edge_l, edge_r, int(strips), int(ny),
                                                       part + size_t(warps) * OBS_COUNT);
    if (cudaPeekAtLastError() != cudaSuccess) return 1;
    *partials = part;
    *rows = warps + eb;
    return 0;
}

}  // namespace qlga

// ===================================================================== tiled 1D step: launch
//
// k_batch_step serves the batches and single 1D lattices alike (tile tables or, for a single
// lattice, tiles computed from the block index).  Its launch shape (threads per CTA, sites per
// thread, tile width = their product) is picked by timing the candidates on the live state.

namespace qlga {

constexpr int kBatchNumWidths = 6;
constexpr int kBatchWidths[kBatchNumWidths] = {32, 64, 128, 256, 120, 248};  // tile widths (sites)

// A launch shape: tile width (index into kBatchWidths) = threads x sites per thread - 8 (steps - 1),
// steps = fused steps per launch (2: temporal blocking, FP32 only).
struct BatchCand {
    int tile, threads, spt, steps;
};
constexpr int kBatchNumCands = 11;
constexpr BatchCand kBatchCands[kBatchNumCands] = {
    {0, 32, 1, 1},  {1, 64, 1, 1},  {2, 128, 1, 1}, {3, 256, 1, 1}, {2, 64, 2, 1},  {3, 128, 2, 1},
    {3, 64, 4, 1},  {5, 64, 4, 2},  {5, 128, 2, 2}, {4, 64, 2, 2},  {5, 256, 1, 2}};
constexpr int kBatchDefaultCand = 1;  // before tuning: 64 threads, one site each

// Candidate index of a shape (threads, sites per thread, steps), -1 if there is none.
inline int batch_cand_of(int threads, int spt, int steps) {
    for (int ci = 0; ci < kBatchNumCands; ++ci)
        if (kBatchCands[ci].threads == threads && kBatchCands[ci].spt == spt && kBatchCands[ci].steps == steps)
            return ci;
    return -1;
}

struct TileArgs {
    cudaStream_t stream;
    int precision, variant;
    bool pot;
    const void* in;
    void* out;
    const BatchTile* tiles;  // nullptr: a single lattice of single_L sites
    int ntiles;
    const BatchRun* runs;
    const void* consts;
    unsigned* status;
    int64_t single_L;
    PotParams single_params;
};

template <class T, int V, bool POT, int W, int SPT, int STEPS>
void tile_launch_shape(const TileArgs& a) {
    constexpr int TOUT = W * SPT - 8 * (STEPS - 1);
    const int nb = a.tiles ? a.ntiles : int((a.single_L + TOUT - 1) / TOUT);
    const PotConst<T> pc = a.tiles ? PotConst<T>() : PotConst<T>(a.single_params);
    k_batch_step<T, V, POT, W, SPT, STEPS><<<nb, W, 0, a.stream>>>(
        static_cast<const T*>(a.in), static_cast<T*>(a.out), a.tiles, a.runs,
        static_cast<const PotConst<T>*>(a.consts), a.status, int(a.single_L), pc);
}

template <class T, int V, bool POT>
void tile_launch_cand(const TileArgs& a, int ci) {
    switch (ci) {
        case 0: tile_launch_shape<T, V, POT, 32, 1, 1>(a); return;
        case 1: tile_launch_shape<T, V, POT, 64, 1, 1>(a); return;
        case 2: tile_launch_shape<T, V, POT, 128, 1, 1>(a); return;
        case 3: tile_launch_shape<T, V, POT, 256, 1, 1>(a); return;
        case 4: tile_launch_shape<T, V, POT, 64, 2, 1>(a); return;
        case 5: tile_launch_shape<T, V, POT, 128, 2, 1>(a); return;
        case 6: tile_launch_shape<T, V, POT, 64, 4, 1>(a); return;
        default: break;
    }
    if constexpr (sizeof(T) == 4 && POT) {  // two steps per launch: FP32 fused steps only
        switch (ci) {
            case 7: tile_launch_shape<T, V, POT, 64, 4, 2>(a); return;
            case 8: tile_launch_shape<T, V, POT, 128, 2, 2>(a); return;
            case 9: tile_launch_shape<T, V, POT, 64, 2, 2>(a); return;
            case 10: tile_launch_shape<T, V, POT, 256, 1, 2>(a); return;
            default: break;
        }
    }
}

// Whether shape ci runs for this precision and kind of launch (two-step shapes: FP32 fused steps).
inline bool tile_cand_ok(int precision, bool pot, int ci) {
    return ci >= 0 && ci < kBatchNumCands && (kBatchCands[ci].steps == 1 || (precision == 32 && pot));
}

// Launch k_batch_step with shape ci (errors left in cudaGetLastError()); ci must pass
// tile_cand_ok.
inline void tile_step_launch(const TileArgs& a, int ci) {
    if (a.precision == 32) {
        if (a.variant == 0) { if (a.pot) tile_launch_cand<float, 0, true>(a, ci); else tile_launch_cand<float, 0, false>(a, ci); }
        else { if (a.pot) tile_launch_cand<float, 1, true>(a, ci); else tile_launch_cand<float, 1, false>(a, ci); }
    } else {
        if (a.variant == 0) { if (a.pot) tile_launch_cand<double, 0, true>(a, ci); else tile_launch_cand<double, 0, false>(a, ci); }
        else { if (a.pot) tile_launch_cand<double, 1, true>(a, ci); else tile_launch_cand<double, 1, false>(a, ci); }
    }
}

}  // namespace qlga

// ===================================================================== handle

struct qlga_handle {
    qlga_config cfg;
    cudaStream_t stream;
    bool owns;
    void* X[2];
    void* tmp;       // one state buffer of work space
    double* partials;
    double* obs_dev;
    unsigned* status;
    int cur;
    bool pending_k;  // buffer holds X with true state K X
    int64_t step;
    int64_t launches;  // kernels launched by this handle
    int tile_cand;  // 1D: launch shape of the tiled step (index into kBatchCands), -1 untuned
    int tile_cand2;  // 1D: two-step shape when it beats tile_cand per step, else -1
    int tile_lanes;   // 1D: fused steps by the lane-parallel kernel with 5 or 10 lanes per site, 0: not
    int step2d_mode;  // QLGA_STEP2D_AUTO / _FUSED / _TWO_PASS
    // CUDA graphs of graph_steps fused steps starting (and ending) on buffer 0 or 1
    int graph_steps;
    int64_t graph_launches;  // kernels in one graph
    cudaGraphExec_t graph[2];
};

namespace {

int64_t nsites_of(const qlga_config& c) { return c.nx * c.ny; }

size_t state_bytes_of(const qlga_config& c) {
    return size_t(nsites_of(c)) * 20 * (c.precision == 32 ? 4 : 8);
}

size_t workspace_bytes_of(const qlga_config& c) {
    return align256(state_bytes_of(c)) + align256(sizeof(double) * kObsMaxBlocks * OBS_COUNT) +
           align256(sizeof(double) * OBS_COUNT) + align256(sizeof(unsigned));
}

qlga_status check_cfg(const qlga_config* c) {
    if (!c) return fail(QLGA_ERR_INVALID_ARG, "config is NULL%s");
    if (c->ndim != 1 && c->ndim != 2) return fail(QLGA_ERR_INVALID_ARG, "ndim must be 1 or 2%s");
    if (c->precision != 32 && c->precision != 64)
        return fail(QLGA_ERR_INVALID_ARG, "precision must be 32 or 64%s");
    if (c->nx < 8) return fail(QLGA_ERR_INVALID_ARG, "nx must be >= 8%s");
    if (c->ndim == 1 && c->ny != 1) return fail(QLGA_ERR_INVALID_ARG, "ny must be 1 for ndim 1%s");
    if (c->ndim == 2 && c->ny < 8) return fail(QLGA_ERR_INVALID_ARG, "ny must be >= 8 for ndim 2%s");
    if (c->nx > (int64_t(1) << 31) || c->ny > (int64_t(1) << 31) || nsites_of(*c) > (int64_t(1) << 34))
        return fail(QLGA_ERR_INVALID_ARG, "lattice too large%s");
    if (!std::isfinite(c->g0) || !std::isfinite(c->g1) || !std::isfinite(c->g2) || !std::isfinite(c->epsilon))
        return fail(QLGA_ERR_INVALID_ARG, "couplings and epsilon must be finite%s");
    if (c->interleave != 0 && c->interleave != 1) return fail(QLGA_ERR_INVALID_ARG, "interleave must be 0 or 1%s");
    if (c->kinetic_variant != QLGA_KINETIC_K1 && c->kinetic_variant != QLGA_KINETIC_K2)
        return fail(QLGA_ERR_INVALID_ARG, "kinetic_variant must be K1 or K2%s");
    return QLGA_OK;
}

// Threads per block for the per-site kernels: 256, or fewer for small lattices so that the grid
// still spreads over every SM (2 blocks per SM), never below one warp.
int block_for(int64_t n) {
    const int64_t b = 2 * int64_t(device_sms());
    int64_t t = (n + b - 1) / b;
    t = (t + 31) / 32 * 32;
    return int(t < 32 ? 32 : (t > kThreads ? kThreads : t));
}

// Grid of a grid-stride per-site kernel: one block per `threads` sites, at most `cap` blocks
// (cap = 0: 16 per SM of the current device).
int grid_for_block(int64_t n, int threads, int cap = 0) {
    if (cap <= 0) cap = 16 * device_sms();
    int64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return int(g < 1 ? 1 : g);
}

int grid_for(int64_t n, int cap = 0) {
    if (cap <= 0) cap = 16 * device_sms();
    int64_t g = (n + kThreads - 1) / kThreads;
    if (g > cap) g = cap;
    return int(g < 1 ? 1 : g);
}

PotParams pot_params(const qlga_config& c, double delta) { return PotParams{c.g0, c.g1, c.g2, delta}; }

template <class T, bool HELD_PQ = false>
qlga_status launch_potential(qlga_handle* h, void* buf, double delta) {
    const int64_t n = nsites_of(h->cfg);
    const int nt = block_for(n);
    k_potential<T, std::is_same<T, float>::value, HELD_PQ><<<grid_for_block(n, nt), nt, 0, h->stream>>>(
        static_cast<T*>(buf), n, PotConst<T>(pot_params(h->cfg, delta)), h->status);
    QLGA_CUDA(cudaGetLastError(), "k_potential launch");
    h->launches += 1;
    return QLGA_OK;
}

template <class T, int V, bool POT>
qlga_status launch_axis_t(qlga_handle* h, const void* in, void* out, int axis) {
    const int64_t n = nsites_of(h->cfg);
    const int nt = block_for(n);
    k_kinetic_axis<T, V, POT><<<grid_for_block(n, nt), nt, 0, h->stream>>>(
        static_cast<const T*>(in), static_cast<T*>(out), h->cfg.nx, h->cfg.ny, axis,
        PotConst<T>(pot_params(h->cfg, 1.0)), h->status);
    QLGA_CUDA(cudaGetLastError(), "k_kinetic_axis launch");
    h->launches += 1;
    return QLGA_OK;
}

qlga_status launch_axis(qlga_handle* h, const void* in, void* out, int axis, bool pot) {
    const bool f = h->cfg.precision == 32;
    const int v = h->cfg.kinetic_variant;
    if (f) {
        if (v == 0) return pot ? launch_axis_t<float, 0, true>(h, in, out, axis) : launch_axis_t<float, 0, false>(h, in, out, axis);
        return pot ? launch_axis_t<float, 1, true>(h, in, out, axis) : launch_axis_t<float, 1, false>(h, in, out, axis);
    }
    if (v == 0) return pot ? launch_axis_t<double, 0, true>(h, in, out, axis) : launch_axis_t<double, 0, false>(h, in, out, axis);
    return pot ? launch_axis_t<double, 1, true>(h, in, out, axis) : launch_axis_t<double, 1, false>(h, in, out, axis);
}

qlga_status launch_pot(qlga_handle* h, void* buf, double delta) {
    return h->cfg.precision == 32 ? launch_potential<float>(h, buf, delta) : launch_potential<double>(h, buf, delta);
}

bool step2d_uses_fused(const qlga_handle* h);

// Whether this handle holds its states pending K in the (P, Q) form: 1D lattices and the fused
// 2D steps (the two-pass 2D form holds (a, bt)).
bool held_pq(const qlga_handle* h) { return h->cfg.ndim == 1 || step2d_uses_fused(h); }

// U on a true state, leaving it held pending K (X = U psi, true state K X): the first half of a
// step, in the form the handle's kinetic pass reads.
qlga_status launch_pot_held(qlga_handle* h, void* buf) {
    if (held_pq(h))
        return h->cfg.precision == 32 ? launch_potential<float, true>(h, buf, 1.0) : launch_potential<double, true>(h, buf, 1.0);
    return launch_pot(h, buf, 1.0);
}

// One interleaved axis pass (U^(1/(4 ndim)) before each of the axis's four blocks), in -> out.
template <class T, int V>
void interleave_launch_t(qlga_handle* h, const void* in, void* out, int axis) {
    const PotConst<T> PC(pot_params(h->cfg, 1.0 / (4.0 * h->cfg.ndim)));
    const int64_t nx = h->cfg.nx, ny = h->cfg.ny;
    if (axis == 0) {
        const int64_t tiles = ((nx + kIlvXTile - 1) / kIlvXTile) * ny;
        const int64_t cap = 16 * int64_t(device_sms());
        const int grid = int(tiles < cap ? tiles : cap);
        k_interleave_x<T, V><<<grid, kIlvXThreads, 0, h->stream>>>(static_cast<const T*>(in), static_cast<T*>(out), nx, ny, PC, h->status);
    } else {
        const int64_t strips = (nx + kIlvYThreads - 1) / kIlvYThreads;
        int64_t chunks = (8 * int64_t(device_sms())) / strips;
        chunks = chunks < 1 ? 1 : (chunks > ny ? ny : chunks);
        k_interleave_y<T, V><<<int(strips * chunks), kIlvYThreads, 0, h->stream>>>(static_cast<const T*>(in), static_cast<T*>(out), nx, ny, int(chunks), PC, h->status);
    }
}

qlga_status launch_interleave(qlga_handle* h, const void* in, void* out, int axis) {
    const bool f = h->cfg.precision == 32;
    if (h->cfg.kinetic_variant == 0) {
        if (f) interleave_launch_t<float, 0>(h, in, out, axis);
        else interleave_launch_t<double, 0>(h, in, out, axis);
    } else {
        if (f) interleave_launch_t<float, 1>(h, in, out, axis);
        else interleave_launch_t<double, 1>(h, in, out, axis);
    }
    QLGA_CUDA(cudaGetLastError(), "interleave launch");
    h->launches += 1;
    return QLGA_OK;
}

// Events that are destroyed when the scope ends, whatever the exit path.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t create() {
        cudaError_t e = cudaEventCreate(&e0);
        return e == cudaSuccess ? cudaEventCreate(&e1) : e;
    }
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Time per step of one kind of launch on the live state: launch(stream, k) issues launch k of a
// run of launches of `steps` fused steps on `stream`; even k step one free buffer into another and
// odd k step back, as the real run alternates its two buffers (launches that all read one buffer
// and write another timed the 1D shapes in a different order than the real run: the tuner chose a
// shape 8% slower than the best on the 16384-site lattice).  Direct: a warm-up launch, then two
// timed ones on `stream`.  Graphed (where the steps will be replayed
// from graphs, which hide the host's launch gaps; such lattices take microseconds per step):
// kTuneGraphSteps steps captured into a graph on the capture stream cs, one warm-up replay, then
// three timed replays.
constexpr int kTuneGraphSteps = 16;
constexpr int kTuneRounds = 2;

template <class Launch>
cudaError_t time_per_step(cudaStream_t stream, cudaStream_t cs, bool graphed, int steps, EventPair& ev,
                          Launch&& launch, float* ms_per_step) {
    cudaError_t e = cudaSuccess;
    float ms = 0.f;
    if (graphed) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < kTuneGraphSteps / steps; ++k) launch(cs, k);
            e = cudaStreamEndCapture(cs, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) e = cudaGraphLaunch(x, stream);  // warm
        if (e == cudaSuccess) e = cudaEventRecord(ev.e0, stream);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaGraphLaunch(x, stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev.e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.e0, ev.e1);
        if (x) cudaGraphExecDestroy(x);
        *ms_per_step = ms / float(3 * kTuneGraphSteps);
    } else {
        launch(stream, 0);  // warm
        e = cudaEventRecord(ev.e0, stream);
        for (int k = 1; k <= 2 && e == cudaSuccess; ++k) launch(stream, k);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev.e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.e0, ev.e1);
        *ms_per_step = ms / float(2 * steps);
    }
    return e;
}

// Times the launch shapes of the tiled kernel (launch(ci, stream, k): launch k of shape ci) with
// time_per_step and compares the time per step.  best1 is the fastest one-step shape (its time
// in *t1); best2 the fastest two-step shape if `two_step` allows them and it beats best1 per step,
// else -1 (*t2 its time, or a large value).  Every shape is timed in kTuneRounds rounds over all
// shapes and keeps its best time, so that one disturbed timing does not decide the choice (single
// rounds picked shapes 7% apart on the same 16384-site lattice from run to run).
template <class Launch>
cudaError_t tune_shapes(cudaStream_t stream, bool two_step, bool graphed, Launch&& launch, int* best1, int* best2,
                        float* t1_out = nullptr, float* t2_out = nullptr) {
    EventPair ev;
    cudaError_t e = ev.create();
    cudaStream_t cs = nullptr;
    if (e == cudaSuccess && graphed) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    float t1 = 1e30f, t2 = 1e30f;
    *best1 = kBatchDefaultCand;
    *best2 = -1;
    float best_ms[kBatchNumCands];
    for (int ci = 0; ci < kBatchNumCands; ++ci) best_ms[ci] = 1e30f;
    for (int round = 0; round < kTuneRounds && e == cudaSuccess; ++round) {
        for (int ci = 0; ci < kBatchNumCands && e == cudaSuccess; ++ci) {
            const int steps = kBatchCands[ci].steps;
            if (steps == 2 && !two_step) continue;
            float ms = 0.f;
            e = time_per_step(stream, cs, graphed, steps, ev, [&](cudaStream_t st, int k) { launch(ci, st, k); }, &ms);
            if (e == cudaSuccess && ms < best_ms[ci]) best_ms[ci] = ms;
        }
    }
    for (int ci = 0; ci < kBatchNumCands && e == cudaSuccess; ++ci) {
        const int steps = kBatchCands[ci].steps;
        if (steps == 2 && !two_step) continue;
        if (steps == 1 && best_ms[ci] < t1) {
            t1 = best_ms[ci];
            *best1 = ci;
        } else if (steps == 2 && best_ms[ci] < t2) {
            t2 = best_ms[ci];
            *best2 = ci;
        }
    }
    if (cs) cudaStreamDestroy(cs);
    if (*best2 >= 0 && !(t2 < t1)) *best2 = -1;
    if (t1_out) *t1_out = t1;
    if (t2_out) *t2_out = t2;
    return e;
}

// Number of kernel launches tune_shapes issues.
inline int tune_launches(bool two_step, bool graphed) {
    int n = 0;
    for (int ci = 0; ci < kBatchNumCands; ++ci) {
        const int steps = kBatchCands[ci].steps;
        if (steps == 2 && !two_step) continue;
        n += graphed ? 4 * (kTuneGraphSteps / steps) : 3;
    }
    return kTuneRounds * n;
}

// One fused step of a single 1D lattice by the lane-parallel kernel (qlga_lanes1d.cuh) with lps
// lanes per site (5 or 10).
template <class T>
void lanes_1d_launch_t(const TileArgs& a, int lps) {
    const PotConst<T> pc(a.single_params);
    const T* in = static_cast<const T*>(a.in);
    T* out = static_cast<T*>(a.out);
    const int L = int(a.single_L);
    const int nb = (L + 30 / lps - 1) / (30 / lps);
    if (lps == 5) {
        if (a.variant == 0) k_step1d_lanes<T, 0, 5><<<nb, 32, 0, a.stream>>>(in, out, L, pc, a.status);
        else k_step1d_lanes<T, 1, 5><<<nb, 32, 0, a.stream>>>(in, out, L, pc, a.status);
    } else {
        if (a.variant == 0) k_step1d_lanes<T, 0, 10><<<nb, 32, 0, a.stream>>>(in, out, L, pc, a.status);
        else k_step1d_lanes<T, 1, 10><<<nb, 32, 0, a.stream>>>(in, out, L, pc, a.status);
    }
}
inline void lanes_1d_launch(const TileArgs& a, int lps) {
    if (a.precision == 32) lanes_1d_launch_t<float>(a, lps);
    else lanes_1d_launch_t<double>(a, lps);
}

// 1D: one fused step (or the kinetic operator alone) of the whole lattice, in -> out; `steps`
// fused steps (2: the two-step shape of the tiled kernel, which the handle has only in FP32 and
// when it is faster).  The first fused step times, on the live state and writing only `out`, the
// tiled kernel's launch shapes (shared with the batches) and the lane-parallel kernel, and keeps
// the fastest per step; read-outs (pot = false) take the fastest one-step shape of the tiled
// kernel.
qlga_status tile_1d(qlga_handle* h, const void* in, void* out, bool pot, int steps = 1) {
    TileArgs a{h->stream, h->cfg.precision, h->cfg.kinetic_variant, pot, in, out, nullptr, 0, nullptr,
               nullptr, h->status, h->cfg.nx, pot_params(h->cfg, 1.0)};
    if (pot && h->tile_cand < 0) {
        const bool two = h->cfg.precision == 32 && !h->cfg.interleave;
        const bool graphed = h->graph_steps > 0;
        float t1 = 0.f, t2 = 0.f, tl = 0.f;
        // the candidates step a copy of the state back and forth between the work buffer and this
        // step's output buffer, both free until the step itself runs
        QLGA_CUDA(cudaMemcpyAsync(h->tmp, in, state_bytes_of(h->cfg), cudaMemcpyDeviceToDevice, h->stream),
                  "1D tuning copy");
        auto alternate = [&](TileArgs& b, cudaStream_t st, int k) {
            b.stream = st;
            b.in = (k & 1) ? out : h->tmp;
            b.out = (k & 1) ? h->tmp : out;
        };
        cudaError_t e = tune_shapes(h->stream, two, graphed,
                                    [&](int ci, cudaStream_t st, int k) {
                                        TileArgs b = a;
                                        alternate(b, st, k);
                                        tile_step_launch(b, ci);
                                    },
                                    &h->tile_cand, &h->tile_cand2, &t1, &t2);
        int lanes = 0;
        // the lane-parallel kernel, 5 and 10 lanes per site, in FP64 (in FP32 it is no faster, and
        // its warp-maximum Taylor degree over 3 or 6 sites instead of 32 lets the FP32 truncation,
        // which accumulates, grow: config 0 after 2000 steps 1.1e-4 against ~1e-5)
        if (e == cudaSuccess && h->cfg.precision == 64) {
            EventPair ev;
            cudaStream_t cs = nullptr;
            e = ev.create();
            if (e == cudaSuccess && graphed) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            for (int lps = 5; lps <= 10 && e == cudaSuccess; lps += 5) {
                e = time_per_step(h->stream, cs, graphed, 1, ev,
                                  [&](cudaStream_t st, int k) {
                                      TileArgs b = a;
                                      alternate(b, st, k);
                                      lanes_1d_launch(b, lps);
                                  },
                                  &tl);
                if (e == cudaSuccess && tl < t1 && (h->tile_cand2 < 0 || tl < t2)) {
                    lanes = lps;
                    t1 = tl;
                    t2 = tl;
                }
            }
            if (cs) cudaStreamDestroy(cs);
        }
        if (e != cudaSuccess) return cuda_fail(e, "1D step tuning");
        h->tile_lanes = lanes;
        if (lanes) h->tile_cand2 = -1;
        h->launches += tune_launches(two, graphed) + (h->cfg.precision == 64 ? 2 * (graphed ? 4 * kTuneGraphSteps : 3) : 0);
    }
    if (pot && steps == 1 && h->tile_lanes) {
        lanes_1d_launch(a, h->tile_lanes);
        QLGA_CUDA(cudaGetLastError(), "k_step1d_lanes launch");
        h->launches += 1;
        return QLGA_OK;
    }
    const int ci = steps == 2 ? h->tile_cand2 : (h->tile_cand >= 0 ? h->tile_cand : kBatchDefaultCand);
    if (!tile_cand_ok(h->cfg.precision, pot, ci)) return fail(QLGA_ERR_INVALID_ARG, "no launch shape for this 1D step%s");
    tile_step_launch(a, ci);
    QLGA_CUDA(cudaGetLastError(), "k_batch_step launch (1D)");
    h->launches += 1;
    return QLGA_OK;
}

// Whether the next fused steps of this handle can go two per launch (1D FP32, tuned or forced).
bool two_step_1d(const qlga_handle* h) {
    return h->cfg.ndim == 1 && !h->cfg.interleave && h->pending_k && h->tile_cand2 >= 0;
}

// The 2D kernel form of this handle's steps (see qlga_set_step2d_mode).
bool step2d_uses_fused(const qlga_handle* h) {
    if (h->cfg.ndim != 2 || !step2d_f32_supported(h->cfg.nx, h->cfg.ny)) return false;
    if (h->step2d_mode == QLGA_STEP2D_FUSED) return true;
    if (h->step2d_mode == QLGA_STEP2D_TWO_PASS) return false;
    return h->cfg.precision == 32 || step2d_f64_fused_preferred(h->cfg.nx, h->cfg.ny);
}

// Apply the full kinetic operator: in -> out (out may not alias in).  2D uses `mid` for the
// x pass.  With pot, U follows the last axis (the fused step).
// out = [U] K in.  held: `in` is a state held pending K (the handle's held form; the fused FP32
// step reads (P, Q)); otherwise a true state in the resident layout, which the two-pass form
// takes on a lattice that holds (P, Q).
qlga_status kinetic_into(qlga_handle* h, const void* in, void* out, void* mid, bool pot, bool held = true) {
    if (h->cfg.ndim == 1) {
        if (!held) {  // a true state: the 1D kernels read (P, Q), so write that form into mid first
            const int64_t np = 5 * nsites_of(h->cfg);
            if (h->cfg.precision == 32)
                k_pq_of_resident<float><<<grid_for(np), kThreads, 0, h->stream>>>(static_cast<const float*>(in), static_cast<float*>(mid), np);
            else
                k_pq_of_resident<double><<<grid_for(np), kThreads, 0, h->stream>>>(static_cast<const double*>(in), static_cast<double*>(mid), np);
            QLGA_CUDA(cudaGetLastError(), "k_pq_of_resident launch");
            h->launches += 1;
            in = mid;
        }
        return tile_1d(h, in, out, pot);
    }
    if (step2d_uses_fused(h) && (held || !held_pq(h))) {
        const int err = h->cfg.precision == 32
            ? step2d_f32_launch(static_cast<const float*>(in), static_cast<float*>(out), h->cfg.nx, h->cfg.ny,
                                h->cfg.kinetic_variant, pot, PotConst<float>(pot_params(h->cfg, 1.0)), h->status,
                                h->stream)
            : step2d_f64_launch(static_cast<const double*>(in), static_cast<double*>(out), h->cfg.nx, h->cfg.ny,
                                h->cfg.kinetic_variant, pot, PotConst<double>(pot_params(h->cfg, 1.0)), h->status,
                                h->stream);
        if (err) return cuda_fail(cudaGetLastError(), "step2d launch");
        h->launches += 1;
        return QLGA_OK;
    }
    qlga_status s = launch_axis(h, in, mid, 0, false);
    if (s != QLGA_OK) return s;
    return launch_axis(h, mid, out, 1, pot);
}

// ABI layout <-> resident layout (see qlga_device.cuh); src may equal dst.
qlga_status launch_convert(qlga_handle* h, const void* src, void* dst, bool to_resident) {
    const int64_t np = 5 * nsites_of(h->cfg);
    const int g = grid_for(np);
    if (h->cfg.precision == 32) {
        if (to_resident)
            k_convert_layout<float, true><<<g, kThreads, 0, h->stream>>>(static_cast<const float*>(src), static_cast<float*>(dst), np);
        else
            k_convert_layout<float, false><<<g, kThreads, 0, h->stream>>>(static_cast<const float*>(src), static_cast<float*>(dst), np);
    } else {
        if (to_resident)
            k_convert_layout<double, true><<<g, kThreads, 0, h->stream>>>(static_cast<const double*>(src), static_cast<double*>(dst), np);
        else
            k_convert_layout<double, false><<<g, kThreads, 0, h->stream>>>(static_cast<const double*>(src), static_cast<double*>(dst), np);
    }
    QLGA_CUDA(cudaGetLastError(), "k_convert_layout launch");
    h->launches += 1;
    return QLGA_OK;
}

// Make the buffer hold the true state (pending K applied).
qlga_status materialize(qlga_handle* h) {
    if (!h->pending_k) return QLGA_OK;
    qlga_status s = kinetic_into(h, h->X[h->cur], h->X[1 - h->cur], h->tmp, false);
    if (s != QLGA_OK) return s;
    h->cur ^= 1;
    h->pending_k = false;
    return QLGA_OK;
}

// Device pointer of the true state without changing the representation.
qlga_status true_state_view(qlga_handle* h, const void** view) {
    if (!h->pending_k) {
        *view = h->X[h->cur];
        return QLGA_OK;
    }
    void* dst = h->cfg.ndim == 1 ? h->tmp : h->X[1 - h->cur];
    qlga_status s = kinetic_into(h, h->X[h->cur], dst, h->tmp, false);
    *view = dst;
    return s;
}

qlga_status check_status_word(qlga_handle* h) {
    unsigned st = 0;
    QLGA_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream), "status read");
    QLGA_CUDA(cudaStreamSynchronize(h->stream), "stream sync");
    if (st & 1u) {
        cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream);
        return fail(QLGA_ERR_NOT_FINITE,
                    "the potential exponent ||delta (V - c)|| exceeded 4 or was not finite: the "
                    "field is too large for the lattice scaling (use a smaller epsilon)%s");
    }
    return QLGA_OK;
}

// Capture (once per buffer parity) and launch a graph of graph_steps fused steps.  The graph
// holds the same launches qlga_step issues one by one; graph_steps is even, so it starts and
// ends on buffer h->cur.
void graphs_release(qlga_handle* h) {
    for (int p = 0; p < 2; ++p) {
        if (h->graph[p]) cudaGraphExecDestroy(h->graph[p]);
        h->graph[p] = nullptr;
    }
}

qlga_status graph_steps_launch(qlga_handle* h) {
    cudaGraphExec_t& exec = h->graph[h->cur];
    if (!exec) {
        cudaStream_t cs = nullptr;
        QLGA_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
        cudaStream_t saved = h->stream;
        const int64_t launches0 = h->launches;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        qlga_status s = QLGA_OK;
        if (e == cudaSuccess) {
            h->stream = cs;
            int c = h->cur;
            // two fused steps per launch where the handle has them (1D FP32), with an even number
            // of launches so that the graph ends on the buffer it starts from
            const int gs = h->graph_steps;
            const int twos = two_step_1d(h) ? (gs % 4 == 0 ? gs / 2 : (gs - 2) / 2) : 0;
            for (int k = 0; k < twos && s == QLGA_OK; ++k) {
                s = tile_1d(h, h->X[c], h->X[1 - c], true, 2);
                c ^= 1;
            }
            for (int k = 2 * twos; k < gs && s == QLGA_OK; ++k) {
                s = kinetic_into(h, h->X[c], h->X[1 - c], h->tmp, true);
                c ^= 1;
            }
            h->stream = saved;
            e = cudaStreamEndCapture(cs, &g);
        }
        h->graph_launches = h->launches - launches0;
        h->launches = launches0;
        cudaStreamDestroy(cs);
        if (s != QLGA_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            exec = nullptr;
            return cuda_fail(e, "step graph capture");
        }
    }
    QLGA_CUDA(cudaGraphLaunch(exec, h->stream), "step graph launch");
    h->launches += h->graph_launches;
    return QLGA_OK;
}

}  // namespace

// ===================================================================== allocation-free observables
//
// Scratch of qlga_observables_noalloc(): kNoAllocRows block partials of OBS_COUNT doubles, then
// the OBS_COUNT results.  Host code must not pass the array's name to a kernel (in host code it
// names a host-side stand-in); the device address comes from cudaGetSymbolAddress, looked up on
// every call, so it stays valid after the caller resets the device and the module is reloaded.

namespace {
constexpr int kNoAllocRows = kObsMaxBlocks;
constexpr size_t kNoAllocDoubles = size_t(kNoAllocRows) * OBS_COUNT + OBS_COUNT;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {

// Device address of the scratch array on the current device.
qlga_status noalloc_scratch(double** addr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(observables scratch)");
    *addr = static_cast<double*>(p);
    return QLGA_OK;
}

}  // namespace

extern "C" qlga_status qlga_observables_noalloc(const qlga_config* cfg, const void* state_device,
                                                const void* ref_state_device, void* stream,
                                                qlga_obs* out) {
    qlga_status s = check_cfg(cfg);
    if (s != QLGA_OK) return s;
    if (!state_device || !out) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    const int64_t n = nsites_of(*cfg);
    // grid-stride reduction: at most kNoAllocRows blocks, one partial row each, whatever the size
    const int blocks = grid_for(n, std::min(kNoAllocRows, 8 * device_sms()));
    double* scratch = nullptr;
    s = noalloc_scratch(&scratch);
    if (s != QLGA_OK) return s;
    double* result = scratch + size_t(kNoAllocRows) * OBS_COUNT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cfg->precision == 32)
        k_observables<float, false><<<blocks, kThreads, 0, st>>>(static_cast<const float*>(state_device),
                                                          static_cast<const float*>(ref_state_device),
                                                          cfg->nx, cfg->ny, cfg->ndim, cfg->g0, cfg->g1,
                                                          cfg->g2, scratch, 0, n);
    else
        k_observables<double, false><<<blocks, kThreads, 0, st>>>(static_cast<const double*>(state_device),
                                                           static_cast<const double*>(ref_state_device),
                                                           cfg->nx, cfg->ny, cfg->ndim, cfg->g0, cfg->g1,
                                                           cfg->g2, scratch, 0, n);
    QLGA_CUDA(cudaGetLastError(), "k_observables launch (no-alloc)");
    k_reduce_partials<<<OBS_COUNT, kReduceThreads, 0, st>>>(scratch, blocks, OBS_COUNT, result);
    QLGA_CUDA(cudaGetLastError(), "k_reduce_partials launch (no-alloc)");
    double o[OBS_COUNT];
    QLGA_CUDA(cudaMemcpyAsync(o, result, sizeof(o), cudaMemcpyDeviceToHost, st), "no-alloc observables copy");
    QLGA_CUDA(cudaStreamSynchronize(st), "no-alloc observables sync");
    std::memset(out, 0, sizeof(*out));
    out->norm_qubit = o[OBS_NORM_QUBIT];
    out->norm_boson = o[OBS_NORM_BOSON];
    for (int m = 0; m < 5; ++m) {
        out->pop[m] = o[OBS_POP0 + m];
        out->magnetisation += double(2 - m) * o[OBS_POP0 + m];
    }
    out->energy = o[OBS_ENERGY];
    out->singlet_re = o[OBS_SINGLET_RE];
    out->singlet_im = o[OBS_SINGLET_IM];
    out->singlet_fraction = o[OBS_RHO2] > 0 ? o[OBS_THETA2] / o[OBS_RHO2] : 0.0;
    out->overlap_re = o[OBS_OVERLAP_RE];
    out->overlap_im = o[OBS_OVERLAP_IM];
    out->step = 0;
    if (!std::isfinite(out->norm_qubit) || !std::isfinite(out->energy))
        return fail(QLGA_ERR_NOT_FINITE, "the state holds NaN or Inf%s");
    return QLGA_OK;
}

// ===================================================================== C ABI

extern "C" {

qlga_status qlga_state_bytes(const qlga_config* cfg, size_t* bytes) {
    qlga_status s = check_cfg(cfg);
    if (s != QLGA_OK) return s;
    if (!bytes) return fail(QLGA_ERR_INVALID_ARG, "bytes is NULL%s");
    *bytes = state_bytes_of(*cfg);
    return QLGA_OK;
}

qlga_status qlga_workspace_bytes(const qlga_config* cfg, size_t* bytes) {
    qlga_status s = check_cfg(cfg);
    if (s != QLGA_OK) return s;
    if (!bytes) return fail(QLGA_ERR_INVALID_ARG, "bytes is NULL%s");
    *bytes = workspace_bytes_of(*cfg);
    return QLGA_OK;
}

static qlga_status init_handle(qlga_handle* h, const qlga_config* cfg, void* stream, void* x0,
                               void* x1, void* ws) {
    h->cfg = *cfg;
    h->stream = static_cast<cudaStream_t>(stream);
    h->X[0] = x0;
    h->X[1] = x1;
    char* w = static_cast<char*>(ws);
    h->tmp = w;
    w += align256(state_bytes_of(*cfg));
    h->partials = reinterpret_cast<double*>(w);
    w += align256(sizeof(double) * kObsMaxBlocks * OBS_COUNT);
    h->obs_dev = reinterpret_cast<double*>(w);
    w += align256(sizeof(double) * OBS_COUNT);
    h->status = reinterpret_cast<unsigned*>(w);
    h->cur = 0;
    h->pending_k = false;
    h->step = 0;
    h->launches = 0;
    // small lattices are bound by launch latency: replay runs of fused steps from a graph
    h->graph_steps = nsites_of(*cfg) <= kGraphMaxSites ? kGraphDefaultSteps : 0;
    h->graph_launches = 0;
    h->graph[0] = h->graph[1] = nullptr;
    h->tile_cand = -1;
    h->tile_cand2 = -1;
    h->tile_lanes = 0;
    h->step2d_mode = QLGA_STEP2D_AUTO;
    QLGA_CUDA(cudaMemsetAsync(h->X[0], 0, state_bytes_of(*cfg), h->stream), "state clear");
    QLGA_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream), "status clear");
    return QLGA_OK;
}

qlga_status qlga_create(const qlga_config* cfg, void* stream, qlga_handle** out) {
    qlga_status s = check_cfg(cfg);
    if (s != QLGA_OK) return s;
    if (!out) return fail(QLGA_ERR_INVALID_ARG, "out is NULL%s");
    *out = nullptr;
    qlga_handle* h = new qlga_handle();
    h->owns = true;
    void *x0 = nullptr, *x1 = nullptr, *ws = nullptr;
    cudaError_t e = cudaMalloc(&x0, state_bytes_of(*cfg));
    if (e == cudaSuccess) e = cudaMalloc(&x1, state_bytes_of(*cfg));
    if (e == cudaSuccess) e = cudaMalloc(&ws, workspace_bytes_of(*cfg));
    if (e != cudaSuccess) {
        cudaFree(x0);
        cudaFree(x1);
        cudaFree(ws);
        delete h;
        cudaGetLastError();
        return cuda_fail(e, "qlga_create cudaMalloc");
    }
    s = init_handle(h, cfg, stream, x0, x1, ws);
    if (s != QLGA_OK) {
        cudaFree(x0);
        cudaFree(x1);
        cudaFree(ws);
        delete h;
        return s;
    }
    *out = h;
    return QLGA_OK;
}

qlga_status qlga_create_external(const qlga_config* cfg, void* stream, void* state0, void* state1,
                                 void* workspace, size_t workspace_bytes, qlga_handle** out) {
    qlga_status s = check_cfg(cfg);
    if (s != QLGA_OK) return s;
    if (!out || !state0 || !state1 || !workspace) return fail(QLGA_ERR_INVALID_ARG, "NULL pointer argument%s");
    if (workspace_bytes < workspace_bytes_of(*cfg)) return fail(QLGA_ERR_INVALID_ARG, "workspace too small%s");
    if ((reinterpret_cast<uintptr_t>(state0) | reinterpret_cast<uintptr_t>(state1) |
         reinterpret_cast<uintptr_t>(workspace)) & 255u)
        return fail(QLGA_ERR_INVALID_ARG, "buffers must be 256-byte aligned%s");
    *out = nullptr;
    qlga_handle* h = new qlga_handle();
    h->owns = false;
    s = init_handle(h, cfg, stream, state0, state1, workspace);
    if (s != QLGA_OK) {
        delete h;
        return s;
    }
    *out = h;
    return QLGA_OK;
}

qlga_status qlga_load_state(qlga_handle* h, const void* src, int where) {
    if (!h || !src) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (where != QLGA_HOST && where != QLGA_DEVICE) return fail(QLGA_ERR_INVALID_ARG, "where must be QLGA_HOST or QLGA_DEVICE%s");
    const size_t nb = state_bytes_of(h->cfg);
    const void* dev_src = src;
    if (where == QLGA_HOST) {
        QLGA_CUDA(cudaMemcpyAsync(h->tmp, src, nb, cudaMemcpyHostToDevice, h->stream), "qlga_load_state copy");
        dev_src = h->tmp;
    }
    qlga_status s = launch_convert(h, dev_src, h->X[h->cur], true);
    if (s != QLGA_OK) return s;
    if (where == QLGA_HOST) QLGA_CUDA(cudaStreamSynchronize(h->stream), "qlga_load_state sync");
    h->pending_k = false;
    h->step = 0;
    return QLGA_OK;
}

qlga_status qlga_load_boson(qlga_handle* h, const void* psi5, int where) {
    if (!h || !psi5) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (where != QLGA_HOST && where != QLGA_DEVICE) return fail(QLGA_ERR_INVALID_ARG, "where must be QLGA_HOST or QLGA_DEVICE%s");
    const size_t nb = state_bytes_of(h->cfg) / 2;  // 5 complex per site
    const void* src = psi5;
    if (where == QLGA_HOST) {
        QLGA_CUDA(cudaMemcpyAsync(h->tmp, psi5, nb, cudaMemcpyHostToDevice, h->stream), "qlga_load_boson copy");
        src = h->tmp;
    }
    const int64_t n = nsites_of(h->cfg);
    if (h->cfg.precision == 32)
        k_load_boson<float><<<grid_for(5 * n), kThreads, 0, h->stream>>>(static_cast<const float*>(src), static_cast<float*>(h->X[h->cur]), n, float(0.5 * h->cfg.epsilon));
    else
        k_load_boson<double><<<grid_for(5 * n), kThreads, 0, h->stream>>>(static_cast<const double*>(src), static_cast<double*>(h->X[h->cur]), n, 0.5 * h->cfg.epsilon);
    QLGA_CUDA(cudaGetLastError(), "k_load_boson launch");
    h->launches += 1;
    if (where == QLGA_HOST) QLGA_CUDA(cudaStreamSynchronize(h->stream), "qlga_load_boson sync");
    h->pending_k = false;
    h->step = 0;
    return QLGA_OK;
}

qlga_status qlga_get_state(qlga_handle* h, void* dst, int where) {
    if (!h || !dst) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (where != QLGA_HOST && where != QLGA_DEVICE) return fail(QLGA_ERR_INVALID_ARG, "where must be QLGA_HOST or QLGA_DEVICE%s");
    const void* view = nullptr;
    qlga_status s = true_state_view(h, &view);
    if (s != QLGA_OK) return s;
    if (where == QLGA_DEVICE) return launch_convert(h, view, dst, false);
    // host: convert into the work buffer (in place when the view already is it), then copy
    s = launch_convert(h, view, h->tmp, false);
    if (s != QLGA_OK) return s;
    QLGA_CUDA(cudaMemcpyAsync(dst, h->tmp, state_bytes_of(h->cfg), cudaMemcpyDeviceToHost, h->stream), "qlga_get_state copy");
    QLGA_CUDA(cudaStreamSynchronize(h->stream), "qlga_get_state sync");
    return check_status_word(h);
}

qlga_status qlga_step(qlga_handle* h, int64_t n) {
    if (!h) return fail(QLGA_ERR_INVALID_ARG, "handle is NULL%s");
    if (n < 0) return fail(QLGA_ERR_INVALID_ARG, "n must be >= 0%s");
    qlga_status s = QLGA_OK;
    for (int64_t i = 0; i < n; ++i) {
        // runs of fused steps on a small lattice replay a captured graph (same kernels, same
        // arguments, one graph launch instead of graph_steps stream launches)
        if (!h->cfg.interleave && h->pending_k && h->graph_steps > 0 && n - i >= h->graph_steps &&
            h->step >= 2) {
            s = graph_steps_launch(h);
            if (s != QLGA_OK) return s;
            h->step += h->graph_steps;
            i += h->graph_steps - 1;
            continue;
        }
        if (two_step_1d(h) && n - i >= 2) {  // two fused steps in one launch
            s = tile_1d(h, h->X[h->cur], h->X[1 - h->cur], true, 2);
            if (s != QLGA_OK) return s;
            h->cur ^= 1;
            h->step += 2;
            ++i;
            continue;
        }
        if (h->cfg.interleave) {
            // U^(1/(4 ndim)) before every kinetic block, blocks I'_2 I'_2 I'_1 I'_1 per axis:
            // one fused pass per axis
            s = materialize(h);
            if (s != QLGA_OK) return s;
            for (int axis = 0; axis < h->cfg.ndim; ++axis) {
                s = launch_interleave(h, h->X[h->cur], h->X[1 - h->cur], axis);
                if (s != QLGA_OK) return s;
                h->cur ^= 1;
            }
        } else if (!h->pending_k) {
            s = launch_pot_held(h, h->X[h->cur]);  // X = U psi, true state K X
            if (s != QLGA_OK) return s;
            h->pending_k = true;
        } else {
            s = kinetic_into(h, h->X[h->cur], h->X[1 - h->cur], h->tmp, true);
            if (s != QLGA_OK) return s;
            h->cur ^= 1;
        }
        h->step += 1;
    }
    return QLGA_OK;
}

qlga_status qlga_apply_potential(qlga_handle* h, double delta) {
    if (!h) return fail(QLGA_ERR_INVALID_ARG, "handle is NULL%s");
    if (!std::isfinite(delta)) return fail(QLGA_ERR_INVALID_ARG, "delta must be finite%s");
    qlga_status s = materialize(h);
    if (s != QLGA_OK) return s;
    return launch_pot(h, h->X[h->cur], delta);
}

qlga_status qlga_apply_kinetic(qlga_handle* h) {
    if (!h) return fail(QLGA_ERR_INVALID_ARG, "handle is NULL%s");
    qlga_status s = materialize(h);
    if (s != QLGA_OK) return s;
    s = kinetic_into(h, h->X[h->cur], h->X[1 - h->cur], h->tmp, false, false);  // a true state
    if (s != QLGA_OK) return s;
    h->cur ^= 1;
    return QLGA_OK;
}

// Partial rows of the observable sums of the handle's true state over the rows [y0, y1) (the
// forward pair of row y1 - 1 reads row y1, or row 0 when y1 == ny), with the optional
// reference state for the overlap: *partials, *rows.
static qlga_status observables_rows_partials(qlga_handle* h, const void* ref_state_device, int64_t y0, int64_t y1,
                                      double** partials, int* rows) {
    const void* view = nullptr;
    qlga_status s = true_state_view(h, &view);
    if (s != QLGA_OK) return s;
    const int64_t s0 = y0 * h->cfg.nx, s1 = y1 * h->cfg.nx;
    const int blocks = grid_for(s1 - s0, obs_blocks_cap());
    if (h->cfg.precision == 32)
        k_observables<float, true><<<blocks, kThreads, 0, h->stream>>>(static_cast<const float*>(view), static_cast<const float*>(ref_state_device),
                                                                 h->cfg.nx, h->cfg.ny, h->cfg.ndim, h->cfg.g0, h->cfg.g1, h->cfg.g2, h->partials, s0, s1);
    else
        k_observables<double, true><<<blocks, kThreads, 0, h->stream>>>(static_cast<const double*>(view), static_cast<const double*>(ref_state_device),
                                                                  h->cfg.nx, h->cfg.ny, h->cfg.ndim, h->cfg.g0, h->cfg.g1, h->cfg.g2, h->partials, s0, s1);
    QLGA_CUDA(cudaGetLastError(), "k_observables launch");
    h->launches += 1;
    *partials = h->partials;
    *rows = blocks;
    return QLGA_OK;
}

// The observables of qlga_obs from the OBS_COUNT sums.
static void fill_obs(const double* o, int64_t step, qlga_obs* out) {
    std::memset(out, 0, sizeof(*out));
    out->norm_qubit = o[OBS_NORM_QUBIT];
    out->norm_boson = o[OBS_NORM_BOSON];
    out->magnetisation = 0.0;
    for (int m = 0; m < 5; ++m) {
        out->pop[m] = o[OBS_POP0 + m];
        out->magnetisation += double(2 - m) * o[OBS_POP0 + m];
    }
    out->energy = o[OBS_ENERGY];
    out->singlet_re = o[OBS_SINGLET_RE];
    out->singlet_im = o[OBS_SINGLET_IM];
    out->singlet_fraction = o[OBS_RHO2] > 0 ? o[OBS_THETA2] / o[OBS_RHO2] : 0.0;
    out->overlap_re = o[OBS_OVERLAP_RE];
    out->overlap_im = o[OBS_OVERLAP_IM];
    out->step = step;
}

// Partial rows of the observable sums of the handle's true state (with the optional reference
// state for the overlap): *partials, *rows.
qlga_status observables_partials(qlga_handle* h, const void* ref_state_device, double** partials, int* rows) {
    if (h->pending_k && h->cfg.precision == 32 && step2d_uses_fused(h)) {
        // one read of the state: K on the fly in the warp strips, the sums in the same pass; the
        // work buffer is free between steps and holds the edge fields and partial rows
        const int err = obs2d_f32_launch(static_cast<const float*>(h->X[h->cur]),
                                         static_cast<const float*>(ref_state_device), h->cfg.nx, h->cfg.ny,
                                         h->cfg.kinetic_variant, h->cfg.g0, h->cfg.g1, h->cfg.g2, h->tmp,
                                         state_bytes_of(h->cfg), h->stream, partials, rows);
        if (err == 1) return cuda_fail(cudaGetLastError(), "k_obs2d_f32 launch");
        if (err == 0) {
            h->launches += 2;
            return QLGA_OK;
        }
    }
    return observables_rows_partials(h, ref_state_device, 0, h->cfg.ny, partials, rows);
}

qlga_status qlga_observables(qlga_handle* h, const void* ref_state_device, qlga_obs* out) {
    if (!h || !out) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    double* partials = nullptr;
    int rows = 0;
    qlga_status s = observables_partials(h, ref_state_device, &partials, &rows);
    if (s != QLGA_OK) return s;
    k_reduce_partials<<<OBS_COUNT, kReduceThreads, 0, h->stream>>>(partials, rows, OBS_COUNT, h->obs_dev);
    QLGA_CUDA(cudaGetLastError(), "k_reduce_partials launch");
    h->launches += 1;
    double o[OBS_COUNT];
    QLGA_CUDA(cudaMemcpyAsync(o, h->obs_dev, sizeof(o), cudaMemcpyDeviceToHost, h->stream), "observables copy");
    QLGA_CUDA(cudaStreamSynchronize(h->stream), "observables sync");
    fill_obs(o, h->step, out);
    s = check_status_word(h);
    if (s != QLGA_OK) return s;
    if (!std::isfinite(out->norm_qubit) || !std::isfinite(out->energy))
        return fail(QLGA_ERR_NOT_FINITE, "the state holds NaN or Inf%s");
    return QLGA_OK;
}

qlga_status qlga_observable_sums(qlga_handle* h, int64_t y0, int64_t y1, const void* ref_state_device,
                                 double* sums) {
    if (!h || !sums) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (y0 < 0 || y1 <= y0 || y1 > h->cfg.ny) return fail(QLGA_ERR_INVALID_ARG, "rows must satisfy 0 <= y0 < y1 <= ny%s");
    double* partials = nullptr;
    int rows = 0;
    qlga_status s = observables_rows_partials(h, ref_state_device, y0, y1, &partials, &rows);
    if (s != QLGA_OK) return s;
    k_reduce_partials<<<OBS_COUNT, kReduceThreads, 0, h->stream>>>(partials, rows, OBS_COUNT, h->obs_dev);
    QLGA_CUDA(cudaGetLastError(), "k_reduce_partials launch");
    h->launches += 1;
    QLGA_CUDA(cudaMemcpyAsync(sums, h->obs_dev, sizeof(double) * OBS_COUNT, cudaMemcpyDeviceToHost, h->stream),
              "observable sums copy");
    QLGA_CUDA(cudaStreamSynchronize(h->stream), "observable sums sync");
    return check_status_word(h);
}

qlga_status qlga_obs_from_sums(const double* sums, int64_t step, qlga_obs* out) {
    if (!sums || !out) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    fill_obs(sums, step, out);
    if (!std::isfinite(out->norm_qubit) || !std::isfinite(out->energy))
        return fail(QLGA_ERR_NOT_FINITE, "the sums hold NaN or Inf%s");
    return QLGA_OK;
}

qlga_status qlga_objective(qlga_handle* h, const void* x_device, int32_t level, const double* g,
                           const double* weights, double* values, double* dg, void* cot_device) {
    if (!h || !x_device || !g || !values) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (level < 0 || level > 4) return fail(QLGA_ERR_INVALID_ARG, "level must be 0..4 (m = +2..-2)%s");
    if ((cot_device || dg) && !weights) return fail(QLGA_ERR_INVALID_ARG, "a cotangent needs the weights%s");
    if (!std::isfinite(g[0]) || !std::isfinite(g[1]) || !std::isfinite(g[2]))
        return fail(QLGA_ERR_INVALID_ARG, "couplings must be finite%s");
    const int64_t n = nsites_of(h->cfg);
    const int blocks = grid_for(n, obs_blocks_cap());  // partial rows of OBJ_COUNT <= OBS_COUNT doubles
    const bool f = h->cfg.precision == 32;
    if (f)
        k_objective_sums<float><<<blocks, kObjThreads, 0, h->stream>>>(static_cast<const float*>(x_device), h->cfg.nx, h->cfg.ny,
                                                                   h->cfg.ndim, level, g[0], g[1], g[2], h->partials);
    else
        k_objective_sums<double><<<blocks, kObjThreads, 0, h->stream>>>(static_cast<const double*>(x_device), h->cfg.nx, h->cfg.ny,
                                                                    h->cfg.ndim, level, g[0], g[1], g[2], h->partials);
    QLGA_CUDA(cudaGetLastError(), "k_objective_sums launch");
    k_reduce_partials<<<OBJ_COUNT, kReduceThreads, 0, h->stream>>>(h->partials, blocks, OBJ_COUNT, h->obs_dev);
    QLGA_CUDA(cudaGetLastError(), "k_reduce_partials launch");
    h->launches += 2;
    if (cot_device) {
        if (f)
            k_objective_cot<float><<<grid_for(n), kObjThreads, 0, h->stream>>>(
                static_cast<const float*>(x_device), static_cast<float*>(cot_device), h->cfg.nx, h->cfg.ny, h->cfg.ndim,
                level, g[0], g[1], g[2], h->obs_dev, weights[0], weights[1], weights[2]);
        else
            k_objective_cot<double><<<grid_for(n), kObjThreads, 0, h->stream>>>(
                static_cast<const double*>(x_device), static_cast<double*>(cot_device), h->cfg.nx, h->cfg.ny, h->cfg.ndim,
                level, g[0], g[1], g[2], h->obs_dev, weights[0], weights[1], weights[2]);
        QLGA_CUDA(cudaGetLastError(), "k_objective_cot launch");
        h->launches += 1;
    }
    double o[OBJ_COUNT];
    QLGA_CUDA(cudaMemcpyAsync(o, h->obs_dev, sizeof(o), cudaMemcpyDeviceToHost, h->stream), "objective sums copy");
    QLGA_CUDA(cudaStreamSynchronize(h->stream), "objective sync");
    values[0] = o[OBJ_POP];
    values[1] = o[OBJ_RHO2] > 0.0 ? o[OBJ_THETA2] / o[OBJ_RHO2] : 0.0;
    values[2] = o[OBJ_ENERGY];
    if (dg) {  // the energy term's explicit dependence on the couplings
        dg[0] = weights[2] * 0.5 * o[OBJ_RHO2];
        dg[1] = weights[2] * 0.5 * o[OBJ_F2];
        dg[2] = weights[2] * 0.1 * o[OBJ_THETA2];
    }
    if (!std::isfinite(values[0]) || !std::isfinite(values[2]))
        return fail(QLGA_ERR_NOT_FINITE, "the state holds NaN or Inf%s");
    return QLGA_OK;
}

static size_t site_bytes_of(const qlga_config& c) { return size_t(c.precision == 32 ? 16 : 32); }

qlga_status qlga_copy_rows(qlga_handle* h, int64_t y0, int64_t nrows, void* buf, int direction) {
    if (!h || !buf) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (direction != QLGA_ROWS_OUT && direction != QLGA_ROWS_IN)
        return fail(QLGA_ERR_INVALID_ARG, "direction must be QLGA_ROWS_OUT or QLGA_ROWS_IN%s");
    if (y0 < 0 || nrows <= 0 || y0 + nrows > h->cfg.ny)
        return fail(QLGA_ERR_INVALID_ARG, "rows must satisfy 0 <= y0 and y0 + nrows <= ny%s");
    const size_t sb = site_bytes_of(h->cfg);
    const size_t plane = size_t(nsites_of(h->cfg)) * sb;
    const size_t width = size_t(nrows) * size_t(h->cfg.nx) * sb;
    char* state = static_cast<char*>(h->X[h->cur]) + size_t(y0) * size_t(h->cfg.nx) * sb;
    if (direction == QLGA_ROWS_OUT)
        QLGA_CUDA(cudaMemcpy2DAsync(buf, width, state, plane, width, 5, cudaMemcpyDefault, h->stream), "qlga_copy_rows out");
    else
        QLGA_CUDA(cudaMemcpy2DAsync(state, plane, buf, width, width, 5, cudaMemcpyDefault, h->stream), "qlga_copy_rows in");
    return QLGA_OK;
}

qlga_status qlga_exchange_rows(qlga_handle* src, int64_t ysrc, qlga_handle* dst, int64_t ydst, int64_t nrows) {
    if (!src || !dst) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (src->cfg.nx != dst->cfg.nx || src->cfg.precision != dst->cfg.precision || src->cfg.ndim != dst->cfg.ndim)
        return fail(QLGA_ERR_INVALID_ARG, "the two handles differ in nx, precision or ndim%s");
    if (src->pending_k != dst->pending_k)
        return fail(QLGA_ERR_INVALID_ARG, "the two handles hold their states in different forms (step them together)%s");
    if (nrows <= 0 || ysrc < 0 || ydst < 0 || ysrc + nrows > src->cfg.ny || ydst + nrows > dst->cfg.ny)
        return fail(QLGA_ERR_INVALID_ARG, "rows outside a lattice%s");
    if (src == dst && ((ysrc < ydst + nrows) && (ydst < ysrc + nrows)))
        return fail(QLGA_ERR_INVALID_ARG, "overlapping rows in one handle%s");
    if (src->stream != dst->stream) {  // the copy waits for the source's queued work
        cudaEvent_t ev = nullptr;
        QLGA_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "exchange event");
        cudaError_t e = cudaEventRecord(ev, src->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(dst->stream, ev, 0);
        cudaEventDestroy(ev);
        QLGA_CUDA(e, "exchange ordering");
    }
    const size_t sb = site_bytes_of(src->cfg);
    const size_t width = size_t(nrows) * size_t(src->cfg.nx) * sb;
    const char* from = static_cast<const char*>(src->X[src->cur]) + size_t(ysrc) * size_t(src->cfg.nx) * sb;
    char* to = static_cast<char*>(dst->X[dst->cur]) + size_t(ydst) * size_t(dst->cfg.nx) * sb;
    QLGA_CUDA(cudaMemcpy2DAsync(to, size_t(nsites_of(dst->cfg)) * sb, from, size_t(nsites_of(src->cfg)) * sb, width, 5,
                                cudaMemcpyDefault, dst->stream),
              "qlga_exchange_rows");
    if (src->stream != dst->stream) {  // the source must not overwrite its rows before the copy ends
        cudaEvent_t ev = nullptr;
        QLGA_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "exchange event");
        cudaError_t e = cudaEventRecord(ev, dst->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(src->stream, ev, 0);
        cudaEventDestroy(ev);
        QLGA_CUDA(e, "exchange ordering");
    }
    return QLGA_OK;
}

qlga_status qlga_fields(qlga_handle* h, void* dst, int where) {
    if (!h || !dst) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (where != QLGA_HOST && where != QLGA_DEVICE) return fail(QLGA_ERR_INVALID_ARG, "where must be QLGA_HOST or QLGA_DEVICE%s");
    const void* view = nullptr;
    qlga_status s = true_state_view(h, &view);
    if (s != QLGA_OK) return s;
    const int64_t n = nsites_of(h->cfg);
    const size_t bytes = size_t(n) * 11 * (h->cfg.precision == 32 ? 4 : 8);  // < one state buffer
    void* target = dst;
    if (where == QLGA_HOST) target = (view == h->tmp) ? h->X[1 - h->cur] : h->tmp;
    if (h->cfg.ndim == 2) {
        const int64_t tiles = ((h->cfg.nx + kFieldsTx - 1) / kFieldsTx) * ((h->cfg.ny + kFieldsTy - 1) / kFieldsTy);
        // one wave of resident blocks: each block loops over tiles, so blocks beyond the resident
        // count would start only when the first wave has finished all of its tiles
        int per_sm = 0;
        QLGA_CUDA(h->cfg.precision == 32
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fields2d<float>, kFieldsTx * kFieldsTy, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fields2d<double>, kFieldsTx * kFieldsTy, 0),
                  "k_fields2d occupancy");
        const int64_t cap = int64_t(per_sm > 0 ? per_sm : 1) * device_sms();
        const int grid = int(tiles < cap ? tiles : cap);
        if (h->cfg.precision == 32)
            k_fields2d<float><<<grid, kFieldsTx * kFieldsTy, 0, h->stream>>>(static_cast<const float*>(view), static_cast<float*>(target), h->cfg.nx, h->cfg.ny);
        else
            k_fields2d<double><<<grid, kFieldsTx * kFieldsTy, 0, h->stream>>>(static_cast<const double*>(view), static_cast<double*>(target), h->cfg.nx, h->cfg.ny);
    } else if (h->cfg.precision == 32) {
        k_fields<float><<<grid_for(n), kThreads, 0, h->stream>>>(static_cast<const float*>(view), static_cast<float*>(target), h->cfg.nx, h->cfg.ny, h->cfg.ndim);
    } else {
        k_fields<double><<<grid_for(n), kThreads, 0, h->stream>>>(static_cast<const double*>(view), static_cast<double*>(target), h->cfg.nx, h->cfg.ny, h->cfg.ndim);
    }
    QLGA_CUDA(cudaGetLastError(), "k_fields launch");
    h->launches += 1;
    if (where == QLGA_HOST) {
        QLGA_CUDA(cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, h->stream), "qlga_fields copy");
        QLGA_CUDA(cudaStreamSynchronize(h->stream), "qlga_fields sync");
    }
    return QLGA_OK;
}

qlga_status qlga_launch_count(const qlga_handle* h, int64_t* count) {
    if (!h || !count) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    *count = h->launches;
    return QLGA_OK;
}

qlga_status qlga_set_graph_steps(qlga_handle* h, int32_t steps) {
    if (!h) return fail(QLGA_ERR_INVALID_ARG, "handle is NULL%s");
    if (steps < 0 || steps % 2 != 0 || steps > 4096) return fail(QLGA_ERR_INVALID_ARG, "graph steps must be even, in 0..4096%s");
    cudaStreamSynchronize(h->stream);
    graphs_release(h);
    h->graph_steps = steps;
    return QLGA_OK;
}

qlga_status qlga_set_step2d_mode(qlga_handle* h, int32_t mode) {
    if (!h) return fail(QLGA_ERR_INVALID_ARG, "handle is NULL%s");
    if (mode != QLGA_STEP2D_AUTO && mode != QLGA_STEP2D_FUSED && mode != QLGA_STEP2D_TWO_PASS)
        return fail(QLGA_ERR_INVALID_ARG, "mode must be QLGA_STEP2D_AUTO, _FUSED or _TWO_PASS%s");
    if (mode == QLGA_STEP2D_FUSED && (h->cfg.ndim != 2 || !step2d_f32_supported(h->cfg.nx, h->cfg.ny)))
        return fail(QLGA_ERR_UNSUPPORTED, "the fused 2D kernel needs a 2D lattice with nx a multiple of 32%s");
    // a state held pending K is read out first: the new form may hold it differently
    qlga_status s = materialize(h);
    if (s != QLGA_OK) return s;
    cudaStreamSynchronize(h->stream);
    graphs_release(h);
    h->step2d_mode = mode;
    return QLGA_OK;
}

qlga_status qlga_get_step2d_kernel(qlga_handle* h, int32_t* kernel) {
    if (!h || !kernel) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    *kernel = h->cfg.ndim != 2 ? 0 : (step2d_uses_fused(h) ? QLGA_STEP2D_FUSED : QLGA_STEP2D_TWO_PASS);
    return QLGA_OK;
}

qlga_status qlga_set_1d_shape(qlga_handle* h, int32_t threads, int32_t sites_per_thread, int32_t steps) {
    if (!h) return fail(QLGA_ERR_INVALID_ARG, "handle is NULL%s");
    if (h->cfg.ndim != 1) return fail(QLGA_ERR_UNSUPPORTED, "launch shapes are for 1D lattices%s");
    int c1 = -1, c2 = -1;
    const int lanes = (threads == 5 || threads == 10) && sites_per_thread == 0 && steps == 1 ? threads : 0;
    if (lanes) {
        c1 = kBatchDefaultCand;  // read-outs of the pending state
    } else if (threads != 0 || sites_per_thread != 0 || steps != 0) {
        const int ci = batch_cand_of(threads, sites_per_thread, steps);
        if (ci < 0) return fail(QLGA_ERR_INVALID_ARG, "not one of the launch shapes%s");
        if (steps == 2 && (h->cfg.precision != 32 || h->cfg.interleave))
            return fail(QLGA_ERR_UNSUPPORTED, "two steps per launch need FP32 plain steps%s");
        c1 = steps == 2 ? batch_cand_of(threads, sites_per_thread, 1) : ci;
        c2 = steps == 2 ? ci : -1;
    }
    cudaStreamSynchronize(h->stream);
    graphs_release(h);
    h->tile_cand = c1;
    h->tile_cand2 = c2;
    h->tile_lanes = lanes;
    return QLGA_OK;
}

qlga_status qlga_get_1d_shape(qlga_handle* h, int32_t* threads, int32_t* sites_per_thread, int32_t* steps) {
    if (!h || !threads || !sites_per_thread || !steps) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (h->tile_lanes) {
        *threads = h->tile_lanes;
        *sites_per_thread = 0;
        *steps = 1;
        return QLGA_OK;
    }
    const int ci = h->tile_cand2 >= 0 ? h->tile_cand2 : h->tile_cand;
    *threads = ci >= 0 ? kBatchCands[ci].threads : 0;
    *sites_per_thread = ci >= 0 ? kBatchCands[ci].spt : 0;
    *steps = ci >= 0 ? kBatchCands[ci].steps : 0;
    return QLGA_OK;
}

qlga_status qlga_synchronize(qlga_handle* h) {
    if (!h) return fail(QLGA_ERR_INVALID_ARG, "handle is NULL%s");
    QLGA_CUDA(cudaStreamSynchronize(h->stream), "qlga_synchronize");
    return check_status_word(h);
}

qlga_status qlga_destroy(qlga_handle* h) {
    if (!h) return QLGA_OK;
    cudaStreamSynchronize(h->stream);
    graphs_release(h);
    if (h->owns) {
        cudaFree(h->X[0]);
        cudaFree(h->X[1]);
        cudaFree(h->tmp);
    }
    delete h;
    return QLGA_OK;
}

const char* qlga_status_string(qlga_status s) {
    switch (s) {
        case QLGA_OK: return "ok";
        case QLGA_ERR_INVALID_ARG: return "invalid argument";
        case QLGA_ERR_OOM: return "out of device memory";
        case QLGA_ERR_CUDA: return "CUDA error";
        case QLGA_ERR_TIMEOUT: return "device wait timed out";
        case QLGA_ERR_NOT_FINITE: return "state not finite";
        case QLGA_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* qlga_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ===================================================================== adjoint (reverse mode)
//
// Workspace of the adjoint calls, each part 256-byte aligned: the cotangent and a second
// cotangent buffer (also the middle buffer of a two-pass 2D kinetic read-out), two buffers for
// the post-potential states of a recomputed segment, the per-block coupling partials and their
// sum, ceil(n / C) checkpoints (true states x_0, x_C, x_2C, ...) and C segment slots (true
// states x_k of the segment being pulled back).  All state-sized parts use the resident layout.

namespace {

constexpr int kAdjMaxBlocks = 1216;  // capacity of the coupling partials (8 per SM on 152 SMs)

struct AdjLayout {
    void* cot;
    void* cot_tmp;
    void* w1;
    void* w2;
    double* partials;
    double* result;
    char* ckpt;
    char* slots;
    size_t state;
    int64_t nck, nslots;
    size_t total;
};

AdjLayout adj_layout(const qlga_config& c, int64_t n, int64_t C, void* base) {
    AdjLayout L{};
    L.state = align256(state_bytes_of(c));
    L.nck = n > 0 ? (n + C - 1) / C : 0;
    L.nslots = n < C ? (n > 0 ? n : 1) : C;
    char* p = static_cast<char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* q = p ? p + off : nullptr;
        off += align256(bytes);
        return q;
    };
    L.cot = take(L.state);
    L.cot_tmp = take(L.state);
    L.w1 = take(L.state);
    L.w2 = take(L.state);
    L.partials = reinterpret_cast<double*>(take(sizeof(double) * 3 * kAdjMaxBlocks));
    L.result = reinterpret_cast<double*>(take(sizeof(double) * 3));
    L.ckpt = take(L.state * size_t(L.nck));
    L.slots = take(L.state * size_t(L.nslots));
    L.total = off;
    return L;
}

qlga_status adj_check(qlga_handle* h, int64_t n, int64_t C, void* ws, size_t ws_bytes, AdjLayout* L) {
    if (!h || !ws) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (h->cfg.interleave) return fail(QLGA_ERR_UNSUPPORTED, "the adjoint covers the plain step only (interleave = 0)%s");
    if (n < 0 || C < 1) return fail(QLGA_ERR_INVALID_ARG, "nsteps must be >= 0 and checkpoint_every >= 1%s");
    if (reinterpret_cast<uintptr_t>(ws) & 255u) return fail(QLGA_ERR_INVALID_ARG, "workspace must be 256-byte aligned%s");
    *L = adj_layout(h->cfg, n, C, ws);
    if (ws_bytes < L->total) return fail(QLGA_ERR_INVALID_ARG, "adjoint workspace too small%s");
    return QLGA_OK;
}

template <class T, int V, bool VJP>
void adj_axis_t(qlga_handle* h, const void* gin, void* gout, const void* X, int axis, double* partials, int blocks) {
    k_adjoint_axis<T, V, VJP><<<blocks, kAdjThreads, 0, h->stream>>>(
        static_cast<const T*>(gin), static_cast<T*>(gout), static_cast<const T*>(X), h->cfg.nx, h->cfg.ny,
        axis, AdjConst<T>(pot_params(h->cfg, 1.0)), partials, h->status);
}

template <class T, bool VJP>
void adj_axis_v(qlga_handle* h, const void* gin, void* gout, const void* X, int axis, double* partials, int blocks) {
    if (h->cfg.kinetic_variant == 0) adj_axis_t<T, 0, VJP>(h, gin, gout, X, axis, partials, blocks);
    else adj_axis_t<T, 1, VJP>(h, gin, gout, X, axis, partials, blocks);
}

qlga_status adj_axis(qlga_handle* h, const void* gin, void* gout, const void* X, int axis, bool vjp, double* partials) {
    const int blocks = grid_for_block(nsites_of(h->cfg), kAdjThreads, std::min(kAdjMaxBlocks, 8 * device_sms()));
    if (h->cfg.precision == 32) {
        if (vjp) adj_axis_v<float, true>(h, gin, gout, X, axis, partials, blocks);
        else adj_axis_v<float, false>(h, gin, gout, X, axis, partials, blocks);
    } else {
        if (vjp) adj_axis_v<double, true>(h, gin, gout, X, axis, partials, blocks);
        else adj_axis_v<double, false>(h, gin, gout, X, axis, partials, blocks);
    }
    QLGA_CUDA(cudaGetLastError(), "k_adjoint_axis launch");
    h->launches += 1;
    return QLGA_OK;
}

// cot <- (d step / d x at x_k)^T cot.  The cotangent lives in *cot; 1D swaps it with *tmp.
qlga_status adj_pullback(qlga_handle* h, void** cot, void** tmp, const void* xk, double* partials) {
    qlga_status s;
    if (h->cfg.ndim == 1) {
        s = adj_axis(h, *cot, *tmp, xk, 0, true, partials);
        if (s != QLGA_OK) return s;
        std::swap(*cot, *tmp);
        return QLGA_OK;
    }
    // K = K_y K_x, so K^dagger = K_x^dagger K_y^dagger: y first, then x with the pull-back of U
    s = adj_axis(h, *cot, *tmp, xk, 1, false, partials);
    if (s != QLGA_OK) return s;
    return adj_axis(h, *tmp, *cot, xk, 0, true, partials);
}

qlga_status adj_finish(qlga_handle* h, const AdjLayout& L, void* cot_res, void* cot_dev, double* dcoup) {
    k_reduce_partials<<<3, kReduceThreads, 0, h->stream>>>(L.partials, kAdjMaxBlocks, 3, L.result);
    QLGA_CUDA(cudaGetLastError(), "k_reduce_partials launch (adjoint)");
    h->launches += 1;
    qlga_status s = launch_convert(h, cot_res, cot_dev, false);
    if (s != QLGA_OK) return s;
    double d[3];
    QLGA_CUDA(cudaMemcpyAsync(d, L.result, sizeof(d), cudaMemcpyDeviceToHost, h->stream), "adjoint result copy");
    QLGA_CUDA(cudaStreamSynchronize(h->stream), "adjoint sync");
    if (dcoup)
        for (int i = 0; i < 3; ++i) dcoup[i] = d[i];
    return check_status_word(h);
}

}  // namespace

extern "C" {

qlga_status qlga_adjoint_workspace_bytes(const qlga_config* cfg, int64_t nsteps, int64_t checkpoint_every,
                                         size_t* bytes) {
    qlga_status s = check_cfg(cfg);
    if (s != QLGA_OK) return s;
    if (!bytes) return fail(QLGA_ERR_INVALID_ARG, "bytes is NULL%s");
    if (nsteps < 0 || checkpoint_every < 1) return fail(QLGA_ERR_INVALID_ARG, "nsteps must be >= 0 and checkpoint_every >= 1%s");
    *bytes = adj_layout(*cfg, nsteps, checkpoint_every, nullptr).total;
    return QLGA_OK;
}

qlga_status qlga_adjoint_step(qlga_handle* h, const void* x_device, void* cot_device, void* workspace,
                              size_t workspace_bytes, double* dcoup) {
    AdjLayout L;
    qlga_status s = adj_check(h, 1, 1, workspace, workspace_bytes, &L);
    if (s != QLGA_OK) return s;
    if (!x_device || !cot_device) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    s = launch_convert(h, x_device, L.slots, true);
    if (s != QLGA_OK) return s;
    s = launch_convert(h, cot_device, L.cot, true);
    if (s != QLGA_OK) return s;
    QLGA_CUDA(cudaMemsetAsync(L.partials, 0, sizeof(double) * 3 * kAdjMaxBlocks, h->stream), "partials clear");
    void *cot = L.cot, *tmp = L.cot_tmp;
    s = adj_pullback(h, &cot, &tmp, L.slots, L.partials);
    if (s != QLGA_OK) return s;
    return adj_finish(h, L, cot, cot_device, dcoup);
}

qlga_status qlga_adjoint_forward(qlga_handle* h, const void* x0_device, int64_t nsteps, int64_t checkpoint_every,
                                 void* workspace, size_t workspace_bytes) {
    AdjLayout L;
    qlga_status s = adj_check(h, nsteps, checkpoint_every, workspace, workspace_bytes, &L);
    if (s != QLGA_OK) return s;
    if (!x0_device) return fail(QLGA_ERR_INVALID_ARG, "x0 is NULL%s");
    s = qlga_load_state(h, x0_device, QLGA_DEVICE);
    if (s != QLGA_OK) return s;
    for (int64_t k = 0; k < nsteps; ++k) {
        if (k % checkpoint_every == 0) {
            const void* view = nullptr;
            s = true_state_view(h, &view);
            if (s != QLGA_OK) return s;
            QLGA_CUDA(cudaMemcpyAsync(L.ckpt + L.state * size_t(k / checkpoint_every), view,
                                      state_bytes_of(h->cfg), cudaMemcpyDeviceToDevice, h->stream),
                      "checkpoint copy");
        }
        s = qlga_step(h, 1);
        if (s != QLGA_OK) return s;
    }
    return QLGA_OK;
}

qlga_status qlga_adjoint_backward(qlga_handle* h, int64_t nsteps, int64_t checkpoint_every, void* workspace,
                                  size_t workspace_bytes, void* cot_device, double* dcoup) {
    AdjLayout L;
    qlga_status s = adj_check(h, nsteps, checkpoint_every, workspace, workspace_bytes, &L);
    if (s != QLGA_OK) return s;
    if (!cot_device) return fail(QLGA_ERR_INVALID_ARG, "cot is NULL%s");
    const size_t nb = state_bytes_of(h->cfg);
    s = launch_convert(h, cot_device, L.cot, true);
    if (s != QLGA_OK) return s;
    QLGA_CUDA(cudaMemsetAsync(L.partials, 0, sizeof(double) * 3 * kAdjMaxBlocks, h->stream), "partials clear");
    void *cot = L.cot, *tmp = L.cot_tmp;
    for (int64_t j = L.nck - 1; j >= 0; --j) {
        const int64_t start = j * checkpoint_every;
        const int64_t len = std::min(nsteps - start, checkpoint_every);
        // recompute x_start .. x_{start+len-1} into the slots from the checkpoint:
        // y = U x (post-potential), x_next = K y, y_next = U K y (one fused launch)
        char* slot0 = L.slots;
        QLGA_CUDA(cudaMemcpyAsync(slot0, L.ckpt + L.state * size_t(j), nb, cudaMemcpyDeviceToDevice, h->stream), "slot copy");
        if (len > 1) {
            void *y = L.w1, *y2 = L.w2;
            QLGA_CUDA(cudaMemcpyAsync(y, slot0, nb, cudaMemcpyDeviceToDevice, h->stream), "segment copy");
            s = launch_pot_held(h, y);
            if (s != QLGA_OK) return s;
            for (int64_t i = 1; i < len; ++i) {
                s = kinetic_into(h, y, L.slots + L.state * size_t(i), tmp, false);
                if (s != QLGA_OK) return s;
                if (i + 1 < len) {
                    s = kinetic_into(h, y, y2, tmp, true);
                    if (s != QLGA_OK) return s;
                    std::swap(y, y2);
                }
            }
        }
        for (int64_t i = len - 1; i >= 0; --i) {
            s = adj_pullback(h, &cot, &tmp, L.slots + L.state * size_t(i), L.partials);
            if (s != QLGA_OK) return s;
        }
    }
    return adj_finish(h, L, cot, cot_device, dcoup);
}

qlga_status qlga_adjoint_run(qlga_handle* h, const void* x0_device, int64_t nsteps, int64_t checkpoint_every,
                             void* workspace, size_t workspace_bytes, void* cot_device, double* dcoup) {
    qlga_status s = qlga_adjoint_forward(h, x0_device, nsteps, checkpoint_every, workspace, workspace_bytes);
    if (s != QLGA_OK) return s;
    return qlga_adjoint_backward(h, nsteps, checkpoint_every, workspace, workspace_bytes, cot_device, dcoup);
}

}  // extern "C"

// ===================================================================== batches of 1D lattices

struct qlga_batch {
    int precision, variant, nruns;
    bool use_graph;
    int64_t total_sites;
    cudaStream_t stream;
    void* X[2];
    void* tmp;
    BatchRun* runs;
    void* consts;             // PotConst<T>[nruns]
    double* g3;               // [nruns][3], device
    double* obs_dev;          // [nruns][OBS_COUNT]
    unsigned* status;
    BatchTile* tiles[kBatchNumWidths];  // tiles of the 1D runs, per tile width
    int ntiles[kBatchNumWidths];
    BatchTile* tiles_pot;     // 128-site tiles over every run (planes of 2D runs flattened)
    int ntiles_pot;
    Run2d* runs2d;            // [nruns] (entries of 1D runs unused)
    WarpTask* tasks;          // warp tasks of the 2D runs
    int ntasks;
    int wsel;                 // index into kBatchCands, -1 before tuning
    int wsel2;                // two-step shape when it beats wsel per step (FP32, 1D runs only), else -1
    int cur;
    bool pending_k;
    int64_t step, launches, graph_steps;
    cudaGraphExec_t graph;
    int graph_cur;            // X index the captured steps start from, -1 if none
    int graph_nsteps, graph_nlaunches;  // steps and kernel launches per graph replay
};

namespace {

size_t batch_state_bytes_of(int precision, int64_t total_sites) {
    return size_t(total_sites) * 20 * (precision == 32 ? 4 : 8);
}

qlga_status check_batch_cfg(const qlga_batch_config* c, int64_t* total) {
    if (!c) return fail(QLGA_ERR_INVALID_ARG, "batch config is NULL%s");
    if (c->precision != 32 && c->precision != 64) return fail(QLGA_ERR_INVALID_ARG, "precision must be 32 or 64%s");
    if (c->nruns < 1 || !c->lengths || !c->couplings) return fail(QLGA_ERR_INVALID_ARG, "nruns >= 1 with lengths and couplings required%s");
    if (c->kinetic_variant != QLGA_KINETIC_K1 && c->kinetic_variant != QLGA_KINETIC_K2)
        return fail(QLGA_ERR_INVALID_ARG, "kinetic_variant must be K1 or K2%s");
    int64_t t = 0;
    for (int r = 0; r < c->nruns; ++r) {
        const int64_t nx = c->lengths[r], ny = c->heights ? c->heights[r] : 1;
        if (ny == 1) {
            if (nx < 8 || nx > (int64_t(1) << 30)) return fail(QLGA_ERR_INVALID_ARG, "1D run lengths must be in [8, 2^30]%s");
        } else {
            if (ny < 8 || nx < kStep2dWarpCols || nx % kStep2dWarpCols != 0 || nx * ny > (int64_t(1) << 30))
                return fail(QLGA_ERR_INVALID_ARG, "2D runs need ny >= 8, nx a multiple of 32 and nx * ny <= 2^30%s");
            if (c->precision != 32) return fail(QLGA_ERR_UNSUPPORTED, "2D runs in a batch are stepped in FP32 only%s");
        }
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(c->couplings[3 * r + k])) return fail(QLGA_ERR_INVALID_ARG, "couplings must be finite%s");
        t += nx * ny;
    }
    if (t > (int64_t(1) << 34)) return fail(QLGA_ERR_INVALID_ARG, "batch too large%s");
    *total = t;
    return QLGA_OK;
}

// One fused step (pot) or the kinetic operator alone: in -> out.  1D runs: the tiled kernel with
// launch shape ci; 2D runs: the warp-strip kernel over the task table.
qlga_status batch_launch(qlga_batch* b, const void* in, void* out, bool pot, int ci) {
    if (b->ntiles[kBatchCands[ci].tile] > 0) {
        const TileArgs a{b->stream, b->precision, b->variant, pot, in, out, b->tiles[kBatchCands[ci].tile],
                         b->ntiles[kBatchCands[ci].tile], b->runs, b->consts, b->status, 0, PotParams{}};
        tile_step_launch(a, ci);
        QLGA_CUDA(cudaGetLastError(), "k_batch_step launch");
        b->launches += 1;
    }
    if (b->ntasks > 0) {
        Step2dDevice dv;
        if (step2d_device(&dv)) return cuda_fail(cudaGetLastError(), "2D batch set-up");
        const int grid = (b->ntasks + kStep2dWarpsPerCta - 1) / kStep2dWarpsPerCta;
        const dim3 blk(kStep2dWarpsPerCta * 32);
        const float* fi = static_cast<const float*>(in);
        float* fo = static_cast<float*>(out);
        const PotConst<float>* pc = static_cast<const PotConst<float>*>(b->consts);
        if (b->variant == 0) {
            if (pot) k_batch_step2d_f32<0, true><<<grid, blk, kStep2dWarpSmemBytes, b->stream>>>(fi, fo, b->tasks, b->ntasks, b->runs2d, pc, b->status);
            else k_batch_step2d_f32<0, false><<<grid, blk, kStep2dWarpSmemBytes, b->stream>>>(fi, fo, b->tasks, b->ntasks, b->runs2d, pc, b->status);
        } else {
            if (pot) k_batch_step2d_f32<1, true><<<grid, blk, kStep2dWarpSmemBytes, b->stream>>>(fi, fo, b->tasks, b->ntasks, b->runs2d, pc, b->status);
            else k_batch_step2d_f32<1, false><<<grid, blk, kStep2dWarpSmemBytes, b->stream>>>(fi, fo, b->tasks, b->ntasks, b->runs2d, pc, b->status);
        }
        QLGA_CUDA(cudaGetLastError(), "k_batch_step2d_f32 launch");
        b->launches += 1;
    }
    return QLGA_OK;
}

// The potential unitary alone, in place (the first step from a raw state): U is local, so it
// runs over 128-site tiles of every run's flattened planes, with the run's constants.
template <class T>
__global__ void __launch_bounds__(kThreads) k_batch_potential(T* X, const BatchTile* __restrict__ tiles,
                                                              const BatchRun* __restrict__ runs,
                                                              const PotConst<T>* __restrict__ consts,
                                                              int W, unsigned* status) {
    const BatchTile tile = tiles[blockIdx.x];
    const BatchRun run = runs[tile.run];
    for (int base = 0; base < W; base += blockDim.x) {
        const int j = tile.start + base + threadIdx.x;
        const int js = j < run.L ? j : run.L - 1;  // lanes past the end repeat a valid site
        cpx<T> a[5], b[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const Pair4<T> p = load_raw_pair(X, run.base + int64_t(m) * run.L + js);
            a[m] = {p.v[0], p.v[1]};
            b[m] = {p.v[3], -p.v[2]};
        }
        const PotConst<T> C = consts[tile.run];
        potential_site<T, sizeof(T) == 4, kZframe64<T>>(a, b, C, T(1), T(0.5), status);
        __syncwarp();
        if (j < run.L) {
            // every run (1D tiles, 2D warp strips) holds its state pending K as (P, Q)
#pragma unroll
            for (int m = 0; m < 5; ++m) store_raw_pq(X, run.base + int64_t(m) * run.L + j, a[m], b[m]);
        }
    }
}

qlga_status batch_potential(qlga_batch* b, void* X) {
    // tiles of 128 sites over every run's planes, 128 threads
    if (b->precision == 32)
        k_batch_potential<float><<<b->ntiles_pot, 128, 0, b->stream>>>(static_cast<float*>(X), b->tiles_pot, b->runs, static_cast<const PotConst<float>*>(b->consts), 128, b->status);
    else
        k_batch_potential<double><<<b->ntiles_pot, 128, 0, b->stream>>>(static_cast<double*>(X), b->tiles_pot, b->runs, static_cast<const PotConst<double>*>(b->consts), 128, b->status);
    QLGA_CUDA(cudaGetLastError(), "k_batch_potential launch");
    b->launches += 1;
    return QLGA_OK;
}

// Time each tile width on the live state (two fused steps into work space; the state itself is
// not advanced) and keep the fastest.
qlga_status batch_tune(qlga_batch* b) {
    if (b->ntiles[0] == 0) {  // no 1D runs: nothing to tune
        b->wsel = kBatchDefaultCand;
        b->wsel2 = -1;
        return QLGA_OK;
    }
    const bool two = b->precision == 32 && b->ntasks == 0;
    // the candidates step a copy of the state back and forth between the work buffer and the other
    // state buffer, as the real run alternates its two buffers
    void* other = b->X[1 - b->cur];
    QLGA_CUDA(cudaMemcpyAsync(b->tmp, b->X[b->cur], batch_state_bytes_of(b->precision, b->total_sites),
                              cudaMemcpyDeviceToDevice, b->stream), "batch tuning copy");
    cudaError_t e = tune_shapes(b->stream, two, b->use_graph,
                                [&](int ci, cudaStream_t st, int k) {
                                    cudaStream_t saved = b->stream;
                                    b->stream = st;
                                    batch_launch(b, (k & 1) ? other : b->tmp, (k & 1) ? b->tmp : other, true, ci);
                                    b->stream = saved;
                                },
                                &b->wsel, &b->wsel2);
    if (e != cudaSuccess) return cuda_fail(e, "batch step tuning");
    return QLGA_OK;
}

// Capture fused steps starting from X[cur] into a graph: two launches, cur -> 1-cur -> cur, of
// the two-step shape (4 steps) or of the one-step shape (2 steps).
qlga_status batch_build_graph(qlga_batch* b) {
    cudaGraph_t g;
    QLGA_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    const int c = b->cur;
    const int ci = b->wsel2 >= 0 ? b->wsel2 : b->wsel;
    const int64_t l0 = b->launches;
    qlga_status s1 = batch_launch(b, b->X[c], b->X[1 - c], true, ci);
    qlga_status s2 = s1 == QLGA_OK ? batch_launch(b, b->X[1 - c], b->X[c], true, ci) : s1;
    b->graph_nlaunches = int(b->launches - l0);
    b->launches = l0;  // counted when replayed
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s2 != QLGA_OK) return s2;
    if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    b->graph_cur = c;
    b->graph_nsteps = 2 * kBatchCands[ci].steps;
    return QLGA_OK;
}

qlga_status batch_materialize_view(qlga_batch* b, const void** view) {
    if (!b->pending_k) {
        *view = b->X[b->cur];
        return QLGA_OK;
    }
    qlga_status s = batch_launch(b, b->X[b->cur], b->tmp, false, b->wsel >= 0 ? b->wsel : kBatchDefaultCand);
    *view = b->tmp;
    return s;
}

}  // namespace

extern "C" {

qlga_status qlga_batch_state_bytes(const qlga_batch_config* cfg, size_t* bytes) {
    int64_t total = 0;
    qlga_status s = check_batch_cfg(cfg, &total);
    if (s != QLGA_OK) return s;
    if (!bytes) return fail(QLGA_ERR_INVALID_ARG, "bytes is NULL%s");
    *bytes = batch_state_bytes_of(cfg->precision, total);
    return QLGA_OK;
}

qlga_status qlga_batch_create(const qlga_batch_config* cfg, void* stream, qlga_batch** out) {
    int64_t total = 0;
    qlga_status s = check_batch_cfg(cfg, &total);
    if (s != QLGA_OK) return s;
    if (!out) return fail(QLGA_ERR_INVALID_ARG, "out is NULL%s");
    *out = nullptr;
    qlga_batch* b = new qlga_batch();
    b->precision = cfg->precision;
    b->variant = cfg->kinetic_variant;
    b->nruns = cfg->nruns;
    b->use_graph = cfg->use_graph != 0 && stream != nullptr;
    b->total_sites = total;
    b->stream = static_cast<cudaStream_t>(stream);
    b->wsel = -1;
    b->wsel2 = -1;
    b->graph_nsteps = 0;
    b->graph_nlaunches = 0;
    b->graph_cur = -1;
    const size_t sb = batch_state_bytes_of(cfg->precision, total);
    std::vector<BatchRun> runs(cfg->nruns);
    std::vector<Run2d> runs2d(cfg->nruns);
    int64_t base = 0;
    for (int r = 0; r < cfg->nruns; ++r) {
        const int64_t nx = cfg->lengths[r], ny = cfg->heights ? cfg->heights[r] : 1;
        runs[r].base = base;
        runs[r].L = int(nx * ny);
        runs[r].ny = int(ny);
        runs2d[r] = Run2d{base, int(nx), int(ny)};
        base += 5 * nx * ny;
    }
    // tile tables of the 1D runs (the tiled kernel), 128-site tiles of every run (the potential)
    std::vector<BatchTile> tiles[kBatchNumWidths], tiles_pot;
    for (int r = 0; r < cfg->nruns; ++r) {
        for (int64_t st = 0; st < runs[r].L; st += 128) tiles_pot.push_back(BatchTile{r, int(st)});
        if (runs[r].ny != 1) continue;
        for (int wi = 0; wi < kBatchNumWidths; ++wi)
            for (int64_t st = 0; st < runs[r].L; st += kBatchWidths[wi]) tiles[wi].push_back(BatchTile{r, int(st)});
    }
    for (int wi = 0; wi < kBatchNumWidths; ++wi) b->ntiles[wi] = int(tiles[wi].size());
    b->ntiles_pot = int(tiles_pot.size());
    // warp tasks of the 2D runs: 32-column strips x row chunks of about `rows` rows, sized so that
    // the tasks fill every SM a few times over
    std::vector<WarpTask> tasks;
    {
        int64_t strip_rows = 0;
        for (int r = 0; r < cfg->nruns; ++r)
            if (runs[r].ny > 1) strip_rows += (runs2d[r].nx / kStep2dWarpCols) * int64_t(runs2d[r].ny);
        const int64_t target = int64_t(device_sms()) * 12 * 2;
        const int64_t rows = std::max<int64_t>(16, (strip_rows + target - 1) / std::max<int64_t>(target, 1));
        for (int r = 0; r < cfg->nruns; ++r) {
            if (runs[r].ny == 1) continue;
            const int ny = runs2d[r].ny;
            const int chunks = int(std::max<int64_t>(1, (ny + rows / 2) / rows));
            for (int c = 0; c < chunks; ++c)
                for (int x0 = 0; x0 < runs2d[r].nx; x0 += kStep2dWarpCols)
                    tasks.push_back(WarpTask{r, x0, int((int64_t(c) * ny) / chunks), int((int64_t(c + 1) * ny) / chunks)});
        }
    }
    b->ntasks = int(tasks.size());
    const size_t cbytes = size_t(cfg->nruns) * (cfg->precision == 32 ? sizeof(PotConst<float>) : sizeof(PotConst<double>));
    cudaError_t e = cudaMalloc(&b->X[0], sb);
    if (e == cudaSuccess) e = cudaMalloc(&b->X[1], sb);
    if (e == cudaSuccess) e = cudaMalloc(&b->tmp, sb);
    if (e == cudaSuccess) e = cudaMalloc(&b->runs, sizeof(BatchRun) * runs.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->consts, cbytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->g3, sizeof(double) * 3 * cfg->nruns);
    if (e == cudaSuccess) e = cudaMalloc(&b->obs_dev, sizeof(double) * OBS_COUNT * cfg->nruns);
    if (e == cudaSuccess) e = cudaMalloc(&b->status, sizeof(unsigned));
    for (int wi = 0; wi < kBatchNumWidths && e == cudaSuccess; ++wi)
        e = cudaMalloc(&b->tiles[wi], sizeof(BatchTile) * std::max<size_t>(1, tiles[wi].size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->tiles_pot, sizeof(BatchTile) * tiles_pot.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->runs2d, sizeof(Run2d) * runs2d.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->tasks, sizeof(WarpTask) * std::max<size_t>(1, tasks.size()));
    if (e != cudaSuccess) {
        qlga_batch_destroy(b);
        cudaGetLastError();
        return cuda_fail(e, "qlga_batch_create cudaMalloc");
    }
    std::vector<PotConst<float>> cf;
    std::vector<PotConst<double>> cd;
    for (int r = 0; r < cfg->nruns; ++r) {
        const PotParams P{cfg->couplings[3 * r], cfg->couplings[3 * r + 1], cfg->couplings[3 * r + 2], 1.0};
        cf.push_back(PotConst<float>(P));
        cd.push_back(PotConst<double>(P));
    }
    e = cudaMemcpy(b->runs, runs.data(), sizeof(BatchRun) * runs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cfg->precision == 32 ? cudaMemcpy(b->consts, cf.data(), cbytes, cudaMemcpyHostToDevice)
                                 : cudaMemcpy(b->consts, cd.data(), cbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->g3, cfg->couplings, sizeof(double) * 3 * cfg->nruns, cudaMemcpyHostToDevice);
    for (int wi = 0; wi < kBatchNumWidths && e == cudaSuccess; ++wi)
        if (!tiles[wi].empty())
            e = cudaMemcpy(b->tiles[wi], tiles[wi].data(), sizeof(BatchTile) * tiles[wi].size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->tiles_pot, tiles_pot.data(), sizeof(BatchTile) * tiles_pot.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->runs2d, runs2d.data(), sizeof(Run2d) * runs2d.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tasks.empty())
        e = cudaMemcpy(b->tasks, tasks.data(), sizeof(WarpTask) * tasks.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->X[0], 0, sb);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        qlga_batch_destroy(b);
        return cuda_fail(e, "qlga_batch_create upload");
    }
    *out = b;
    return QLGA_OK;
}

qlga_status qlga_batch_load_state(qlga_batch* b, const void* src, int where) {
    if (!b || !src) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (where != QLGA_HOST && where != QLGA_DEVICE) return fail(QLGA_ERR_INVALID_ARG, "where must be QLGA_HOST or QLGA_DEVICE%s");
    const size_t nb = batch_state_bytes_of(b->precision, b->total_sites);
    const void* dev_src = src;
    if (where == QLGA_HOST) {
        QLGA_CUDA(cudaMemcpyAsync(b->tmp, src, nb, cudaMemcpyHostToDevice, b->stream), "qlga_batch_load_state copy");
        dev_src = b->tmp;
    }
    const int64_t np = 5 * b->total_sites;
    if (b->precision == 32)
        k_convert_layout<float, true><<<grid_for(np), kThreads, 0, b->stream>>>(static_cast<const float*>(dev_src), static_cast<float*>(b->X[b->cur]), np);
    else
        k_convert_layout<double, true><<<grid_for(np), kThreads, 0, b->stream>>>(static_cast<const double*>(dev_src), static_cast<double*>(b->X[b->cur]), np);
    QLGA_CUDA(cudaGetLastError(), "k_convert_layout launch");
    b->launches += 1;
    if (where == QLGA_HOST) QLGA_CUDA(cudaStreamSynchronize(b->stream), "qlga_batch_load_state sync");
    b->pending_k = false;
    b->step = 0;
    return QLGA_OK;
}

qlga_status qlga_batch_get_state(qlga_batch* b, void* dst, int where) {
    if (!b || !dst) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    if (where != QLGA_HOST && where != QLGA_DEVICE) return fail(QLGA_ERR_INVALID_ARG, "where must be QLGA_HOST or QLGA_DEVICE%s");
    const void* view = nullptr;
    qlga_status s = batch_materialize_view(b, &view);
    if (s != QLGA_OK) return s;
    const int64_t np = 5 * b->total_sites;
    void* target = where == QLGA_DEVICE ? dst : b->tmp;
    if (b->precision == 32)
        k_convert_layout<float, false><<<grid_for(np), kThreads, 0, b->stream>>>(static_cast<const float*>(view), static_cast<float*>(target), np);
    else
        k_convert_layout<double, false><<<grid_for(np), kThreads, 0, b->stream>>>(static_cast<const double*>(view), static_cast<double*>(target), np);
    QLGA_CUDA(cudaGetLastError(), "k_convert_layout launch");
    b->launches += 1;
    if (where == QLGA_HOST) {
        QLGA_CUDA(cudaMemcpyAsync(dst, b->tmp, batch_state_bytes_of(b->precision, b->total_sites), cudaMemcpyDeviceToHost, b->stream), "qlga_batch_get_state copy");
        QLGA_CUDA(cudaStreamSynchronize(b->stream), "qlga_batch_get_state sync");
    }
    return QLGA_OK;
}

qlga_status qlga_batch_step(qlga_batch* b, int64_t n) {
    if (!b) return fail(QLGA_ERR_INVALID_ARG, "batch is NULL%s");
    if (n < 0) return fail(QLGA_ERR_INVALID_ARG, "n must be >= 0%s");
    qlga_status s = QLGA_OK;
    while (n > 0) {
        if (!b->pending_k) {
            s = batch_potential(b, b->X[b->cur]);  // X = U psi, true state K X
            if (s != QLGA_OK) return s;
            b->pending_k = true;
            b->step += 1;
            n -= 1;
            continue;
        }
        if (b->wsel < 0) {
            s = batch_tune(b);
            if (s != QLGA_OK) return s;
        }
        const int64_t per_replay = b->wsel2 >= 0 ? 4 : 2;
        if (b->use_graph && n >= per_replay && b->graph_cur < 0) {
            s = batch_build_graph(b);
            if (s != QLGA_OK) return s;
        }
        if (b->use_graph && n >= b->graph_nsteps && b->graph_cur == b->cur) {
            QLGA_CUDA(cudaGraphLaunch(b->graph, b->stream), "graph launch");
            b->launches += b->graph_nlaunches;
            b->graph_steps += b->graph_nsteps;
            b->step += b->graph_nsteps;
            n -= b->graph_nsteps;
            continue;
        }
        const int steps = (b->wsel2 >= 0 && n >= 2) ? 2 : 1;
        s = batch_launch(b, b->X[b->cur], b->X[1 - b->cur], true, steps == 2 ? b->wsel2 : b->wsel);
        if (s != QLGA_OK) return s;
        b->cur ^= 1;
        b->step += steps;
        n -= steps;
    }
    return QLGA_OK;
}

qlga_status qlga_batch_observables(qlga_batch* b, qlga_obs* out) {
    if (!b || !out) return fail(QLGA_ERR_INVALID_ARG, "NULL argument%s");
    const void* view = nullptr;
    qlga_status s = batch_materialize_view(b, &view);
    if (s != QLGA_OK) return s;
    if (b->precision == 32)
        k_batch_observables<float><<<b->nruns, kThreads, 0, b->stream>>>(static_cast<const float*>(view), b->runs, b->g3, b->obs_dev);
    else
        k_batch_observables<double><<<b->nruns, kThreads, 0, b->stream>>>(static_cast<const double*>(view), b->runs, b->g3, b->obs_dev);
    QLGA_CUDA(cudaGetLastError(), "k_batch_observables launch");
    b->launches += 1;
    std::vector<double> o(size_t(b->nruns) * OBS_COUNT);
    QLGA_CUDA(cudaMemcpyAsync(o.data(), b->obs_dev, sizeof(double) * o.size(), cudaMemcpyDeviceToHost, b->stream), "batch observables copy");
    QLGA_CUDA(cudaStreamSynchronize(b->stream), "batch observables sync");
    unsigned st = 0;
    QLGA_CUDA(cudaMemcpy(&st, b->status, sizeof(unsigned), cudaMemcpyDeviceToHost), "batch status read");
    bool finite = true;
    for (int r = 0; r < b->nruns; ++r) {
        const double* q = o.data() + size_t(r) * OBS_COUNT;
        qlga_obs* p = out + r;
        std::memset(p, 0, sizeof(*p));
        p->norm_qubit = q[OBS_NORM_QUBIT];
        p->norm_boson = q[OBS_NORM_BOSON];
        for (int m = 0; m < 5; ++m) {
            p->pop[m] = q[OBS_POP0 + m];
            p->magnetisation += double(2 - m) * q[OBS_POP0 + m];
        }
        p->energy = q[OBS_ENERGY];
        p->singlet_re = q[OBS_SINGLET_RE];
        p->singlet_im = q[OBS_SINGLET_IM];
        p->singlet_fraction = q[OBS_RHO2] > 0 ? q[OBS_THETA2] / q[OBS_RHO2] : 0.0;
        p->step = b->step;
        finite = finite && std::isfinite(p->norm_qubit) && std::isfinite(p->energy);
    }
    if (st & 1u) {
        cudaMemset(b->status, 0, sizeof(unsigned));
        return fail(QLGA_ERR_NOT_FINITE, "the potential exponent exceeded its range in some run%s");
    }
    if (!finite) return fail(QLGA_ERR_NOT_FINITE, "a run's state holds NaN or Inf%s");
    return QLGA_OK;
}

qlga_status qlga_batch_info(const qlga_batch* b, int32_t* tile_width, int32_t* sites_per_thread, int64_t* launches,
                            int64_t* graph_steps, int32_t* steps_per_launch) {
    if (!b) return fail(QLGA_ERR_INVALID_ARG, "batch is NULL%s");
    const int ci = b->wsel2 >= 0 ? b->wsel2 : b->wsel;
    if (tile_width) *tile_width = ci >= 0 ? kBatchWidths[kBatchCands[ci].tile] : 0;
    if (sites_per_thread) *sites_per_thread = ci >= 0 ? kBatchCands[ci].spt : 0;
    if (steps_per_launch) *steps_per_launch = ci >= 0 ? kBatchCands[ci].steps : 0;
    if (launches) *launches = b->launches;
    if (graph_steps) *graph_steps = b->graph_steps;
    return QLGA_OK;
}

qlga_status qlga_batch_set_shape(qlga_batch* b, int32_t threads, int32_t sites_per_thread, int32_t steps) {
    if (!b) return fail(QLGA_ERR_INVALID_ARG, "batch is NULL%s");
    int w1 = -1, w2 = -1;
    if (threads != 0 || sites_per_thread != 0 || steps != 0) {
        const int ci = batch_cand_of(threads, sites_per_thread, steps);
        if (ci < 0) return fail(QLGA_ERR_INVALID_ARG, "not one of the launch shapes%s");
        if (steps == 2 && (b->precision != 32 || b->ntasks > 0))
            return fail(QLGA_ERR_UNSUPPORTED, "two steps per launch need an FP32 batch of 1D runs%s");
        w1 = steps == 2 ? batch_cand_of(threads, sites_per_thread, 1) : ci;
        w2 = steps == 2 ? ci : -1;
    }
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_cur = -1;
    b->graph_nsteps = 0;
    b->wsel = w1;
    b->wsel2 = w2;
    return QLGA_OK;
}

qlga_status qlga_batch_destroy(qlga_batch* b) {
    if (!b) return QLGA_OK;
    if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
    if (b->graph_cur >= 0) cudaGraphExecDestroy(b->graph);
    cudaFree(b->X[0]);
    cudaFree(b->X[1]);
    cudaFree(b->tmp);
    cudaFree(b->runs);
    cudaFree(b->consts);
    cudaFree(b->g3);
    cudaFree(b->obs_dev);
    cudaFree(b->status);
    for (int wi = 0; wi < kBatchNumWidths; ++wi) cudaFree(b->tiles[wi]);
    cudaFree(b->tiles_pot);
    cudaFree(b->runs2d);
    cudaFree(b->tasks);
    delete b;
    return QLGA_OK;
}

}  // extern "C"
