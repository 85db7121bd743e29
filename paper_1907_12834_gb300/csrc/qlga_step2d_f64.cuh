// qlga_step2d_f64.cuh -- fused 2D FP64 QLGA step: one pass over the state per step.
//
// The FP64 form of the warp-strip step of qlga_step2d.cuh: a warp owns 32 columns and a row
// range, stages rows (plus the 4-column periodic halo) in its own cp.async ring, applies the
// nine-point x stencil from shared memory, runs the four y blocks as a register pipeline, then
// the potential unitary, and stores the site.  In FP64 every arithmetic instruction occupies the
// FP64 pipe (2 FMA per SM per cycle on GB300), so the y pipeline -- 8 collides of 4 additions per
// level instead of a second nine-point stencil -- and the single pass are what matter, and so
// does the held form: states pending K are stored as (P, Q) = (a + bt, a - bt) as in FP32, whose
// x stencil has 24 nonzero integer taps per level against 32 in (a, bt); zero taps are skipped at
// compile time and +-1 taps are additions.
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"
#include "qlga_interleave.cuh"  // ilv_stream / ilv_collide (streaming blocks on cpx<T>)
#include "qlga_step2d.cuh"      // cp.async helpers, strip geometry

namespace qlga {

// Store a pair (a, b) as (P, Q) = (a + i b, a - i b) at pair index `pair` of the resident layout
// (two double2; the FP32 form is one float4, pq_of in qlga_step2d.cuh).
__device__ __forceinline__ void put_pq(double* X, int64_t pair, cpx<double> a, cpx<double> b) {
    double2* p = reinterpret_cast<double2*>(X) + 2 * pair;
    p[0] = make_double2(a.re - b.im, a.im + b.re);
    p[1] = make_double2(a.re + b.im, a.im - b.re);
}

// acc + c x for a compile-time integer c (0: nothing, +-1: an addition)
template <int C>
__device__ __forceinline__ double tap64(double x, double acc) {
    if constexpr (C == 0) return acc;
    else if constexpr (C == 1) return acc + x;
    else if constexpr (C == -1) return acc - x;
    else return fma(double(C), x, acc);
}

// One tap of the x stencil on a staged (P, Q) pair (re and im of each).
template <int VARIANT, int K>
__device__ __forceinline__ void stencil_tap64(const double2 P, const double2 Q, cpx<double>& xa, cpx<double>& xbt) {
    constexpr KinStencil S = kStencilPQ[VARIANT];
    xa.re = tap64<S.g[0][1][K]>(Q.x, tap64<S.g[0][0][K]>(P.x, xa.re));
    xa.im = tap64<S.g[0][1][K]>(Q.y, tap64<S.g[0][0][K]>(P.y, xa.im));
    xbt.re = tap64<S.g[1][1][K]>(Q.x, tap64<S.g[1][0][K]>(P.x, xbt.re));
    xbt.im = tap64<S.g[1][1][K]>(Q.y, tap64<S.g[1][0][K]>(P.y, xbt.im));
}

constexpr int kStep2d64WarpsPerCta = 2;
constexpr int kStep2d64SmemBytes =
    kStep2d64WarpsPerCta * kStep2dStages * 5 * kStep2dWarpRowSites * 32;  // double pairs

template <int VARIANT, bool POT>
__global__ void __launch_bounds__(kStep2d64WarpsPerCta * 32)
    k_step2d_f64(const double* __restrict__ in, double* __restrict__ out, int nx, int ny, int chunks,
                 PotConst<double> PC, unsigned* status) {
    extern __shared__ double2 dring[];  // [warp][kStages][5][kStep2dWarpRowSites][2]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int strips = nx / kStep2dWarpCols;
    const int gw = blockIdx.x * kStep2d64WarpsPerCta + w;
    if (gw >= strips * chunks) return;  // whole warp: no block-wide barrier follows
    const int strip = gw % strips;
    const int chunk = gw / strips;
    const int x0 = strip * kStep2dWarpCols;
    const int y_begin = int((int64_t(chunk) * ny) / chunks);
    const int y_end = int((int64_t(chunk + 1) * ny) / chunks);
    const int64_t nsites = int64_t(nx) * ny;
    const double2* in2 = reinterpret_cast<const double2*>(in);
    double2* out2 = reinterpret_cast<double2*>(out);
    double2* ring = dring + w * (kStep2dStages * 5 * kStep2dWarpRowSites * 2);

    const int nrows = (y_end - y_begin) + 8;
    int xm = x0 - kStep2dHalo + lane;
    xm = xm < 0 ? xm + nx : xm;
    int xh = x0 + kStep2dWarpCols - kStep2dHalo + lane;
    xh = xh >= nx ? xh - nx : xh;
    xh = xh >= nx ? xh - nx : xh;
    auto issue_row = [&](int r) {
        int y = y_begin - kStep2dHalo + r;
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        double2* dst = ring + (r % kStep2dStages) * (5 * kStep2dWarpRowSites * 2);
        const double2* src = in2 + 2 * int64_t(y) * nx;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            double2* d = dst + 2 * (m * kStep2dWarpRowSites + lane);
            const double2* g = src + 2 * (m * nsites + xm);
            cp_async_16(d, g);
            cp_async_16(d + 1, g + 1);
        }
        if (lane < 2 * kStep2dHalo) {
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                double2* d = dst + 2 * (m * kStep2dWarpRowSites + kStep2dWarpCols + lane);
                const double2* g = src + 2 * (m * nsites + xh);
                cp_async_16(d, g);
                cp_async_16(d + 1, g + 1);
            }
        }
    };

#pragma unroll
    for (int r = 0; r < kStep2dStages - 1; ++r) {
        if (r < nrows) issue_row(r);
        cp_async_commit();
    }

    cpx<double> yo[4][5], wc[4][5];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m < 5; ++m) yo[k][m] = wc[k][m] = {0.0, 0.0};

    for (int r = 0; r < nrows; ++r) {
        cp_async_wait<kStep2dStages - 2>();
        __syncwarp();
        if (r + kStep2dStages - 1 < nrows) issue_row(r + kStep2dStages - 1);
        cp_async_commit();

        const double2* row = ring + (r % kStep2dStages) * (5 * kStep2dWarpRowSites * 2);
        cpx<double> oa[5], ob[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            // x axis: nine-point stencil (x16, unnormalised) from the held (P, Q) pairs to (a, bt)
            cpx<double> xa = {0.0, 0.0}, xbt = {0.0, 0.0};
            const double2* p = row + 2 * (m * kStep2dWarpRowSites + lane);
            stencil_tap64<VARIANT, 0>(p[0], p[1], xa, xbt);
            stencil_tap64<VARIANT, 1>(p[2], p[3], xa, xbt);
            stencil_tap64<VARIANT, 2>(p[4], p[5], xa, xbt);
            stencil_tap64<VARIANT, 3>(p[6], p[7], xa, xbt);
            stencil_tap64<VARIANT, 4>(p[8], p[9], xa, xbt);
            stencil_tap64<VARIANT, 5>(p[10], p[11], xa, xbt);
            stencil_tap64<VARIANT, 6>(p[12], p[13], xa, xbt);
            stencil_tap64<VARIANT, 7>(p[14], p[15], xa, xbt);
            stencil_tap64<VARIANT, 8>(p[16], p[17], xa, xbt);
            // y axis: I'_2 I'_2 then I'_1 I'_1 as a streaming pipeline (x16, unnormalised)
            ilv_stream<double, VARIANT>(1, xa, xbt, yo[0][m], wc[0][m]);
            ilv_stream<double, VARIANT>(1, xa, xbt, yo[1][m], wc[1][m]);
            ilv_stream<double, VARIANT>(0, xa, xbt, yo[2][m], wc[2][m]);
            ilv_stream<double, VARIANT>(0, xa, xbt, yo[3][m], wc[3][m]);
            oa[m] = xa;
            ob[m] = {xbt.im, -xbt.re};  // b = -i bt
        }
        if (r >= 8) {  // pipeline full: this is output row y_begin + r - 8
            if (POT) {
                potential_site<double, false, kZframe64<double>>(oa, ob, PC, 1.0 / 65536.0, 0.5 / 256.0, status);
            } else {
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    oa[m] = (1.0 / 256.0) * oa[m];
                    ob[m] = (1.0 / 256.0) * ob[m];
                }
            }
            const int64_t site = int64_t(y_begin + r - 8) * nx + x0 + lane;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                if (POT) {  // held pending K again, as (P, Q)
                    put_pq(out, int64_t(m) * nsites + site, oa[m], ob[m]);
                } else {  // the true state, in the resident layout (a, bt = i b)
                    double2* p = out2 + 2 * (int64_t(m) * nsites + site);
                    p[0] = make_double2(oa[m].re, oa[m].im);
                    p[1] = make_double2(-ob[m].im, ob[m].re);
                }
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace qlga
