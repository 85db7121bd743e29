// qlga_step2d_f64.cuh -- fused 2D FP64 QLGA step: one pass over the state per step.
//
// The FP64 form of the warp-strip step of qlga_step2d.cuh: a warp owns 32 columns and a row
// range, stages rows (plus the 4-column periodic halo) in its own cp.async ring, applies the
// nine-point x stencil from shared memory, runs the four y blocks as a register pipeline, then
// the potential unitary, and stores the site.  In FP64 every arithmetic instruction occupies the
// FP64 pipe (2 FMA per SM per cycle on GB300), so the y pipeline -- 8 collides of 4 additions per
// level instead of a second nine-point stencil -- and the single pass are what matter.
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"
#include "qlga_interleave.cuh"  // ilv_stream / ilv_collide (streaming blocks on cpx<T>)
#include "qlga_step2d.cuh"      // cp.async helpers, strip geometry

namespace qlga {

constexpr int kStep2d64WarpsPerCta = 2;
constexpr int kStep2d64SmemBytes =
    kStep2d64WarpsPerCta * kStep2dStages * 5 * kStep2dWarpRowSites * 32;  // double pairs

template <int VARIANT, bool POT>
__global__ void __launch_bounds__(kStep2d64WarpsPerCta * 32)
    k_step2d_f64(const double* __restrict__ in, double* __restrict__ out, int nx, int ny, int chunks,
                 PotConst<double> PC, unsigned* status) {
    extern __shared__ double2 dring[];  // [warp][kStages][5][kStep2dWarpRowSites][2]
    constexpr KinStencil S = kStencil[VARIANT];
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
            // x axis: nine-point stencil (x16, unnormalised) in the (a, bt) basis
            cpx<double> xa = {0.0, 0.0}, xbt = {0.0, 0.0};
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const double2 pa = row[2 * (m * kStep2dWarpRowSites + lane + k)];
                const double2 pb = row[2 * (m * kStep2dWarpRowSites + lane + k) + 1];
                const double caa = S.g[0][0][k], cab = S.g[0][1][k];
                const double cba = S.g[1][0][k], cbb = S.g[1][1][k];
                xa.re = fma(caa, pa.x, fma(cab, pb.x, xa.re));
                xa.im = fma(caa, pa.y, fma(cab, pb.y, xa.im));
                xbt.re = fma(cba, pa.x, fma(cbb, pb.x, xbt.re));
                xbt.im = fma(cba, pa.y, fma(cbb, pb.y, xbt.im));
            }
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
            for (int m = 0; m < 5; ++m) {  // resident layout: (a, bt = i b)
                double2* p = out2 + 2 * (int64_t(m) * nsites + site);
                p[0] = make_double2(oa[m].re, oa[m].im);
                p[1] = make_double2(-ob[m].im, ob[m].re);
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace qlga
