// qlga_obs2d.cuh -- observables of a 2D FP32 lattice held pending K, in one read of the state.
//
// Between steps the library holds X with the true state K X (Sec. VII.B: a run is K (U K)^(n-1)
// U, so each step is one fused pass).  The observables of Sec. III.B (qubit and boson norms,
// populations, energy, singlet amplitude and fraction, overlap) need the true state; the fused
// read-out below applies K with the warp-strip machinery of the fused step (strip_kinetic_rows)
// and, instead of storing K X, sums the per-site terms in compensated FP32 per-lane sums.
//
// The energy's gradient term pairs every site with its +x and +y neighbours (forward
// differences, periodic).  Along y each warp starts one row above its row chunk, so the pair
// (y - 1, y) of every output row y lies inside the warp (row y - 1's field is kept in registers).
// Along x the pair (x, x + 1) lies inside the warp's strip for lanes 0..30 (the next lane's field
// by shuffle); lane 31's pair reaches into the next strip, so lanes 0 and 31 store their field in
// two edge buffers and k_obs2d_edges adds those pairs.  Each warp writes one row of partial sums,
// each edge block one more, and k_reduce_partials adds the rows in a fixed order (deterministic).
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"
#include "qlga_obs.cuh"
#include "qlga_step2d.cuh"

namespace qlga {

constexpr int kObs2dEdgeThreads = 256;
constexpr int kObs2dEdgeBlocksMax = 608;  // 4 per SM on 152 SMs

// Field of edge site (strip, y) in an edge buffer of float2 [strips][ny][5].
__device__ __forceinline__ int64_t obs2d_edge_index(int strip, int y, int ny, int m) {
    return (int64_t(strip) * ny + y) * 5 + m;
}

// Warp gw takes strip gw % strips of row chunk gw / strips (as the fused step) and writes
// partials[gw][OBS_COUNT].  hg0 = g0 / 2, hg1 = g1 / 2, tg2 = g2 / 10 (the energy density's
// coefficients); with REF, ref (ABI layout) gives the overlap sums.  The terms are formed from
// the unnormalised K X (256 times the true field, so the field psi = a + b is 256 psi_true) and
// each sum is scaled once at the end by the power of 1/256 of its degree (exact in binary); the
// qubit norm is the sum of the populations.
template <int VARIANT, bool REF, int STYLE = QLGA_STEP2D_STYLE>
__global__ void __launch_bounds__(kStep2dWarpsPerCta * 32, 3)
    k_obs2d_f32(const float* __restrict__ in, const float* __restrict__ ref, int nx, int ny, int chunks,
                float hg0, float hg1, float tg2, float2* __restrict__ edge_l, float2* __restrict__ edge_r,
                double* __restrict__ partials) {
    extern __shared__ float4 wring[];  // [warp][kStages][5][kStep2dWarpRowSites]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int strips = nx / kStep2dWarpCols;
    const int gw = blockIdx.x * kStep2dWarpsPerCta + w;
    if (gw >= strips * chunks) return;  // whole warp: no block-wide barrier follows
    const int strip = gw % strips;
    const int chunk = gw / strips;
    const int y_begin = int((int64_t(chunk) * ny) / chunks);
    const int y_end = int((int64_t(chunk + 1) * ny) / chunks);
    const int x0 = strip * kStep2dWarpCols;
    const int64_t nsites = int64_t(nx) * ny;
    const float s2 = 1.0f / 65536.0f;  // (1/256)^2: quartic terms to the quadratic scale

    ThreadSum<float> acc[OBS_COUNT];  // OBS_NORM_QUBIT unused (sum of the populations)
    cpx<float> prev[5];               // the field of the previous output row at this lane's column
    strip_kinetic_rows<VARIANT, STYLE>(
        in, nx, ny, x0, y_begin - 1, y_end, wring + w * (kStep2dStages * 5 * kStep2dWarpRowSites), lane,
        [&](int y, cpx<float>(&oa)[5], cpx<float>(&ob)[5]) {
            cpx<float> psi[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) psi[m] = oa[m] + ob[m];
            if (y >= y_begin) {  // warp-uniform; row y_begin - 1 only seeds prev
                float rho = 0.f, grad = 0.f;
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    acc[OBS_POP0 + m].add(norm2(oa[m]) + norm2(ob[m]));
                    rho += norm2(psi[m]);
                    // +x pair inside the strip: (x, x + 1) from the next lane
                    const cpx<float> nb = {__shfl_down_sync(0xffffffffu, psi[m].re, 1),
                                           __shfl_down_sync(0xffffffffu, psi[m].im, 1)};
                    if (lane < kStep2dWarpCols - 1) grad += norm2(nb - psi[m]);
                    // +y pair (y - 1, y)
                    grad += norm2(psi[m] - prev[m]);
                }
                acc[OBS_NORM_BOSON].add(rho);
                float F2;
                cpx<float> th;
                obs_local(psi, F2, th);
                const float th2 = norm2(th);
                acc[OBS_ENERGY].add(grad + s2 * (hg0 * rho * rho + hg1 * F2 + tg2 * th2));
                acc[OBS_SINGLET_RE].add(th.re);
                acc[OBS_SINGLET_IM].add(th.im);
                acc[OBS_THETA2].add(th2);
                acc[OBS_RHO2].add(rho * rho);
                if (REF) {
                    const int64_t site = int64_t(y) * nx + x0 + lane;
                    cpx<float> ov = {0.f, 0.f};
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        cpx<float> a, b;
                        load_pair_abi<float>(ref, nsites, m, site, a, b);
                        ov = cfmac(psi[m], a + b, ov);
                    }
                    acc[OBS_OVERLAP_RE].add(ov.re);
                    acc[OBS_OVERLAP_IM].add(ov.im);
                }
                if (lane == 0 || lane == kStep2dWarpCols - 1) {
                    float2* e = lane == 0 ? edge_l : edge_r;
#pragma unroll
                    for (int m = 0; m < 5; ++m)
                        e[obs2d_edge_index(strip, y, ny, m)] = make_float2(psi[m].re, psi[m].im);
                }
            }
#pragma unroll
            for (int m = 0; m < 5; ++m) prev[m] = psi[m];
        });
    // degree of each sum in the field: 2 (norms, populations, energy at the quadratic scale,
    // singlet amplitude), 4 (theta^2, rho^2), 1 (overlap with the true-scale reference)
    const double q2 = 1.0 / 65536.0, q4 = q2 * q2, q1 = 1.0 / 256.0;
    double pops = 0.0;
#pragma unroll
    for (int k = 0; k < OBS_COUNT; ++k) {
        if (k == OBS_NORM_QUBIT || (!REF && (k == OBS_OVERLAP_RE || k == OBS_OVERLAP_IM))) continue;
        const double v = warp_sum(acc[k].value());
        if (k >= OBS_POP0 && k < OBS_POP0 + 5) pops += v;
        const double sc = (k == OBS_THETA2 || k == OBS_RHO2) ? q4
                          : (k == OBS_OVERLAP_RE || k == OBS_OVERLAP_IM) ? q1
                          : (k == OBS_SINGLET_RE || k == OBS_SINGLET_IM) ? q2 * 0.44721359549995793928  // 1/sqrt(5)
                                                                          : q2;
        if (lane == 0) partials[int64_t(gw) * OBS_COUNT + k] = v * sc;
    }
    if (lane == 0) {
        partials[int64_t(gw) * OBS_COUNT + OBS_NORM_QUBIT] = pops * q2;
        if (!REF) {
            partials[int64_t(gw) * OBS_COUNT + OBS_OVERLAP_RE] = 0.0;
            partials[int64_t(gw) * OBS_COUNT + OBS_OVERLAP_IM] = 0.0;
        }
    }
}

// The x pairs across strip edges: (column 32 s + 31, column 32 (s + 1)), the last strip's pair
// wrapping to column 0.  Each block writes one partial row (energy only).
__global__ void __launch_bounds__(kObs2dEdgeThreads)
    k_obs2d_edges(const float2* __restrict__ edge_l, const float2* __restrict__ edge_r, int strips, int ny,
                  double* __restrict__ partials) {
    ThreadSum<float> acc;
    const int64_t n = int64_t(strips) * ny;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int s = int(i / ny), y = int(i - int64_t(s) * ny);
        const int sn = s + 1 == strips ? 0 : s + 1;
        float grad = 0.f;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const float2 r = edge_l[obs2d_edge_index(sn, y, ny, m)], l = edge_r[obs2d_edge_index(s, y, ny, m)];
            grad += norm2(cpx<float>{r.x - l.x, r.y - l.y});
        }
        acc.add(grad);
    }
    // the edge fields are 256 times the true field
    __shared__ double sh[kObs2dEdgeThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double v = warp_sum(acc.value());
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x < OBS_COUNT) {
        double e = 0.0;
        if (threadIdx.x == OBS_ENERGY)
            for (int k = 0; k < kObs2dEdgeThreads / 32; ++k) e += sh[k];
        partials[int64_t(blockIdx.x) * OBS_COUNT + threadIdx.x] = e * (1.0 / 65536.0);
    }
}

}  // namespace qlga
