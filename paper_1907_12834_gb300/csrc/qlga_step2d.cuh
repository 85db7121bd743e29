// qlga_step2d.cuh -- fused 2D FP32 QLGA step: one HBM read and one HBM write of the state.
//
// out = U(K X) K X with K = K_y K_x (the kinetic blocks I'_1 I'_1 I'_2 I'_2 along x, then along
// y; Sec. VII.B) and U the potential unitary, for a state held "pending K" (see qlga.cu).
//
// Work decomposition ("y-marching warp strips").  A warp owns a strip of 32 columns and a
// contiguous range of output rows; lane l owns column x0 + l and walks down the rows:
//   1. input rows (the 32 columns plus the 4-column x halo on each side, periodic) are staged
//      into the warp's own kStages-deep shared-memory ring with 16-byte cp.async copies, several
//      rows ahead of use; warps synchronise only within themselves (__syncwarp), never with each
//      other, and the halo columns are read by both neighbouring warps (from L2);
//   2. x axis: the nine-point stencil of one axis (integer coefficients derived at compile time
//      from the block definition, taken in the (P, Q) = (a + bt, a - bt) basis the held state is
//      stored in: 24 taps per level instead of 32) reads the lane's column and its 8 neighbours
//      from shared memory;
//   3. y axis: the four blocks I'_2 I'_2 I'_1 I'_1 run as a streaming pipeline down the column:
//      each block keeps one row of history (the unshifted qubit after the first collide and the
//      shifted qubit after the second), so the y axis costs 8 collides of 4 additions per level,
//      has no halo recomputation, and lags the input by 4 rows;
//   4. the potential unitary acts on the finished site, and the site is written as (P, Q) with five
//      16-byte stores that are coalesced across the warp.
// The first 8 rows of a range only fill the pipeline (the dependency cone is +-4 rows).
//
// The kinetic arithmetic is unnormalised: every collide drops its scalar prefactor, so the site
// reaching the potential is 256 (2^8, exact) times the true value; the potential folds the factor
// into its quadratic forms and its output scale.
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"

namespace qlga {

constexpr int kStep2dStages = 4;   // shared-memory ring depth (rows in flight)
constexpr int kStep2dHalo = 4;

__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Packed FP32 pairs: a complex number (re, im) is one float2 and every kinetic coefficient is
// real, so the stencil and the collides act on both halves with one f32x2 instruction.
// STYLE selects how integer coefficients are issued: 0 = f32x2 with coefficient pairs,
// 1 = f32x2 add / sub for +-1 and scalar FFMA with an immediate for larger coefficients,
// 2 = scalar FP32 only.
#ifndef QLGA_STEP2D_STYLE
#define QLGA_STEP2D_STYLE 1
#endif

__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

template <int STYLE>
__device__ __forceinline__ float2 p_add(float2 a, float2 b) {
    if (STYLE == 2) return make_float2(a.x + b.x, a.y + b.y);
    return __fadd2_rn(a, b);
}
template <int STYLE>
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
    if (STYLE == 2) return make_float2(a.x - b.x, a.y - b.y);
    if (STYLE == 1) return f2_sub(a, b);
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
template <int STYLE>
__device__ __forceinline__ float2 p_fma(float c, float2 x, float2 acc) {
    if (STYLE == 0) return __ffma2_rn(make_float2(c, c), x, acc);
    return make_float2(fmaf(c, x.x, acc.x), fmaf(c, x.y, acc.y));
}

// Streaming state of one kinetic block for one level: the unshifted qubit of the first collide
// from the previous row (yo) and the shifted qubit of the second collide from the previous row
// (wc), both in the (a, bt = i b) basis.
struct BlockState {
    float2 yo, wc;
};

// One block I'_c on the stream: input row n (xa, xbt) -> output row n-1, in place.
// c = 1 shifts bt (qubit 2), c = 0 shifts a (qubit 1).  FIRST selects the first collide:
// 0 = [[1, 1], [-1, 1]] (K1), 1 = [[1, -1], [1, 1]] (K2); the second collide is always
// [[1, 1], [-1, 1]].
//
// Z(n-1) takes the shifted qubit from the current row's first collide (S^T: c(j) <- c(j+1)) and the
// other qubit from the previous row (yo); its second collide is W(n-1); the output row takes the
// shifted qubit from W(n-2) (S: c(j) <- c(j-1), held in wc) and the other from W(n-1).  The new yo
// is formed from the inputs only after the old one has been used, so that the loop-carried value
// can keep its register from row to row (5% faster fused step than forming it first).
template <int C, int FIRST, int STYLE>
__device__ __forceinline__ void stream_block(float2& xa, float2& xbt, BlockState& s) {
    const float2 ia = xa, ibt = xbt;
    if (C == 1) {
        const float2 ybt = FIRST == 0 ? p_sub<STYLE>(ibt, ia) : p_add<STYLE>(ia, ibt);
        const float2 wa = p_add<STYLE>(s.yo, ybt), wbt = p_sub<STYLE>(ybt, s.yo);
        s.yo = FIRST == 0 ? p_add<STYLE>(ia, ibt) : p_sub<STYLE>(ia, ibt);
        xa = wa;
        xbt = s.wc;
        s.wc = wbt;
    } else {
        const float2 ya = FIRST == 0 ? p_add<STYLE>(ia, ibt) : p_sub<STYLE>(ia, ibt);
        const float2 wa = p_add<STYLE>(ya, s.yo), wbt = p_sub<STYLE>(s.yo, ya);
        s.yo = FIRST == 0 ? p_sub<STYLE>(ibt, ia) : p_add<STYLE>(ia, ibt);
        xa = s.wc;
        xbt = wbt;
        s.wc = wa;
    }
}

// acc += c * x for a compile-time integer coefficient (0: nothing, +-1: add / subtract)
template <int COEF, int STYLE>
__device__ __forceinline__ float2 tap(float2 x, float2 acc) {
    if (COEF == 0) return acc;
    if (COEF == 1) return p_add<STYLE>(acc, x);
    if (COEF == -1) return p_sub<STYLE>(acc, x);
    return p_fma<STYLE>(float(COEF), x, acc);
}

// A 2D state held pending K on the fused path (FP32 and FP64) stores each pair as
// (P, Q) = (a + bt, a - bt) instead of (a, bt).  With (a, bt) = ((P + Q) / 2, (P - Q) / 2) the nine-point x stencil acting
// on (P, Q) has the integer taps M_k = g_k [[1, 1], [1, -1]] / 2 (every g_k has entries of equal
// parity in each row, so the halves are exact): 24 nonzero taps per level instead of 32 in the
// (a, bt) basis, the fewest of any small integer basis.  The output of the x axis is (a, bt) as
// before; the store of a step converts back to (P, Q).
constexpr KinStencil make_stencil_pq(int variant) {
    const KinStencil g = make_stencil(variant);
    KinStencil S{};
    for (int dst = 0; dst < 2; ++dst)
        for (int k = 0; k < 9; ++k) {
            S.g[dst][0][k] = (g.g[dst][0][k] + g.g[dst][1][k]) / 2;  // coefficient of P
            S.g[dst][1][k] = (g.g[dst][0][k] - g.g[dst][1][k]) / 2;  // coefficient of Q
        }
    return S;
}
constexpr bool stencil_pq_exact(int variant) {
    const KinStencil g = make_stencil(variant);
    for (int dst = 0; dst < 2; ++dst)
        for (int k = 0; k < 9; ++k)
            if ((g.g[dst][0][k] + g.g[dst][1][k]) % 2 != 0) return false;
    return true;
}
static_assert(stencil_pq_exact(0) && stencil_pq_exact(1), "the (P, Q) stencil taps must be integers");
constexpr KinStencil kStencilPQ[2] = {make_stencil_pq(0), make_stencil_pq(1)};

// (P, Q) of a pair (a, b): P = a + i b, Q = a - i b, as one float4
__device__ __forceinline__ float4 pq_of(cpx<float> a, cpx<float> b) {
    return make_float4(a.re - b.im, a.im + b.re, a.re + b.im, a.im - b.re);
}

// One tap of the x stencil on a staged (P, Q) pair.
template <int VARIANT, int K, int STYLE>
__device__ __forceinline__ void stencil_tap(const float4 v, float2& xa, float2& xbt) {
    constexpr KinStencil S = kStencilPQ[VARIANT];
    const float2 P = make_float2(v.x, v.y), Q = make_float2(v.z, v.w);
    xa = tap<S.g[0][0][K], STYLE>(P, xa);
    xa = tap<S.g[0][1][K], STYLE>(Q, xa);
    xbt = tap<S.g[1][0][K], STYLE>(P, xbt);
    xbt = tap<S.g[1][1][K], STYLE>(Q, xbt);
}

// Launch geometry: warps of 32 columns, 4 warps per CTA, each warp with its own ring.
constexpr int kStep2dWarpCols = 32;
constexpr int kStep2dWarpRowSites = kStep2dWarpCols + 2 * kStep2dHalo;  // 40
constexpr int kStep2dWarpsPerCta = 4;
constexpr int kStep2dWarpSmemBytes =
    kStep2dWarpsPerCta * kStep2dStages * 5 * kStep2dWarpRowSites * 16;

// The kinetic operator K on one warp's strip: columns [x0, x0 + 32) of an nx x ny lattice (one
// column per lane), output rows [y_begin, y_end) in order (y_begin may be -1: rows wrap
// periodically); `ring` is the warp's shared-memory ring.  For each output row y it calls
// row_out(y, a, b) with the lane's site of K X as (a, b) pairs, unnormalised: 256 times the true
// value (the eight collides of the two axes drop their factor 1/2 each).
template <int VARIANT, int STYLE, class RowOut>
__device__ __forceinline__ void strip_kinetic_rows(const float* __restrict__ in, int nx, int ny, int x0,
                                                   int y_begin, int y_end, float4* ring, int lane,
                                                   RowOut&& row_out) {
    const int64_t nsites = int64_t(nx) * ny;
    const float4* in4 = reinterpret_cast<const float4*>(in);

    const int nrows = (y_end - y_begin) + 8;
    // ring column r holds lattice column x0 - 4 + r (periodic); lane l stages r = l and, for
    // l < 8, r = 32 + l
    int xm = x0 - kStep2dHalo + lane;
    xm = xm < 0 ? xm + nx : xm;
    int xh = x0 + kStep2dWarpCols - kStep2dHalo + lane;
    xh = xh >= nx ? xh - nx : xh;
    xh = xh >= nx ? xh - nx : xh;  // nx = 32: the right halo wraps onto the strip itself
    auto issue_row = [&](int r) {
        int y = y_begin - kStep2dHalo + r;
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        float4* dst = ring + (r % kStep2dStages) * (5 * kStep2dWarpRowSites);
        const float4* src = in4 + int64_t(y) * nx;
#pragma unroll
        for (int m = 0; m < 5; ++m) cp_async_16(dst + m * kStep2dWarpRowSites + lane, src + m * nsites + xm);
        if (lane < 2 * kStep2dHalo) {
#pragma unroll
            for (int m = 0; m < 5; ++m)
                cp_async_16(dst + m * kStep2dWarpRowSites + kStep2dWarpCols + lane, src + m * nsites + xh);
        }
    };

#pragma unroll
    for (int r = 0; r < kStep2dStages - 1; ++r) {
        if (r < nrows) issue_row(r);
        cp_async_commit();
    }

    BlockState st[5][4];
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int k = 0; k < 4; ++k) st[m][k] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};

    for (int r = 0; r < nrows; ++r) {
        cp_async_wait<kStep2dStages - 2>();
        __syncwarp();
        if (r + kStep2dStages - 1 < nrows) issue_row(r + kStep2dStages - 1);
        cp_async_commit();

        const float4* row = ring + (r % kStep2dStages) * (5 * kStep2dWarpRowSites);
        cpx<float> oa[5], ob[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const float4* p = row + m * kStep2dWarpRowSites + lane;
            float2 xa = make_float2(0.f, 0.f), xbt = make_float2(0.f, 0.f);
            float2 ya = make_float2(0.f, 0.f), ybt = make_float2(0.f, 0.f);
            stencil_tap<VARIANT, 0, STYLE>(p[0], xa, xbt);
            stencil_tap<VARIANT, 1, STYLE>(p[1], ya, ybt);
            stencil_tap<VARIANT, 2, STYLE>(p[2], xa, xbt);
            stencil_tap<VARIANT, 3, STYLE>(p[3], ya, ybt);
            stencil_tap<VARIANT, 4, STYLE>(p[4], xa, xbt);
            stencil_tap<VARIANT, 5, STYLE>(p[5], ya, ybt);
            stencil_tap<VARIANT, 6, STYLE>(p[6], xa, xbt);
            stencil_tap<VARIANT, 7, STYLE>(p[7], ya, ybt);
            stencil_tap<VARIANT, 8, STYLE>(p[8], xa, xbt);
            xa = p_add<STYLE>(xa, ya);
            xbt = p_add<STYLE>(xbt, ybt);
            stream_block<1, VARIANT, STYLE>(xa, xbt, st[m][0]);
            stream_block<1, VARIANT, STYLE>(xa, xbt, st[m][1]);
            stream_block<0, VARIANT, STYLE>(xa, xbt, st[m][2]);
            stream_block<0, VARIANT, STYLE>(xa, xbt, st[m][3]);
            oa[m] = {xa.x, xa.y};
            ob[m] = {xbt.y, -xbt.x};
        }
        if (r >= 8) row_out(y_begin + r - 8, oa, ob);  // pipeline full: output row y_begin + r - 8
    }
    cp_async_wait<0>();
}

// One warp's share of a step: K on the strip (input held pending K as (P, Q)), then (POT) the
// potential unitary and the store of rows [y_begin, y_end) as (P, Q) again.  POT = false stores
// K X alone, the true state, in the resident layout (a, bt).
template <int VARIANT, bool POT, int STYLE>
__device__ __forceinline__ void step2d_strip(const float* __restrict__ in, float* __restrict__ out, int nx,
                                             int ny, int x0, int y_begin, int y_end, const PotConst<float>& PC,
                                             unsigned* status, float4* ring, int lane) {
    const int64_t nsites = int64_t(nx) * ny;
    float4* out4 = reinterpret_cast<float4*>(out);
    strip_kinetic_rows<VARIANT, STYLE>(
        in, nx, ny, x0, y_begin, y_end, ring, lane, [&](int y, cpx<float>(&oa)[5], cpx<float>(&ob)[5]) {
            if (POT) {
                // d = a - b takes the degree of psi: one warp-uniform Horner loop over both vectors
                // runs faster here than a separate, per-lane degree for d (fewer branches)
                potential_site<float, false, true>(oa, ob, PC, 1.0f / 65536.0f, 0.5f / 256.0f, status);
            } else {
                const float s = 1.0f / 256.0f;
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    oa[m] = s * oa[m];
                    ob[m] = s * ob[m];
                }
            }
            const int64_t site = int64_t(y) * nx + x0 + lane;
#pragma unroll
            for (int m = 0; m < 5; ++m)  // POT: held pending K again, as (P, Q); else the true state
                out4[int64_t(m) * nsites + site] =
                    POT ? pq_of(oa[m], ob[m]) : make_float4(oa[m].re, oa[m].im, -ob[m].im, ob[m].re);
        });
}

// The kernel.  POT = false applies the kinetic operator alone (out = K X), used to read out a
// state held pending K.  Warp gw of the grid takes strip gw % strips of row chunk gw / strips.
// The input is always a state held pending K, stored as (P, Q).
template <int VARIANT, bool POT = true, int STYLE = QLGA_STEP2D_STYLE>
__global__ void __launch_bounds__(kStep2dWarpsPerCta * 32, 3)
    k_step2d_f32(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int chunks,
                 PotConst<float> PC, unsigned* status) {
    extern __shared__ float4 wring[];  // [warp][kStages][5][kStep2dWarpRowSites]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int strips = nx / kStep2dWarpCols;
    const int gw = blockIdx.x * kStep2dWarpsPerCta + w;
    if (gw >= strips * chunks) return;  // whole warp: no block-wide barrier follows
    const int strip = gw % strips;
    const int chunk = gw / strips;
    const int y_begin = int((int64_t(chunk) * ny) / chunks);
    const int y_end = int((int64_t(chunk + 1) * ny) / chunks);
    step2d_strip<VARIANT, POT, STYLE>(in, out, nx, ny, strip * kStep2dWarpCols, y_begin, y_end, PC, status,
                                      wring + w * (kStep2dStages * 5 * kStep2dWarpRowSites), lane);
}

// A batch of 2D lattices: warp gw takes task gw of the table -- a run (its state at pair offset
// base, nx x ny sites, constants consts[run]), a strip and a row range.
struct WarpTask {
    int run;
    int x0;
    int y_begin, y_end;
};
struct Run2d {
    int64_t base;  // pair index of plane 0, site 0 of the run
    int nx, ny;
};

template <int VARIANT, bool POT = true, int STYLE = QLGA_STEP2D_STYLE>
__global__ void __launch_bounds__(kStep2dWarpsPerCta * 32, 3)
    k_batch_step2d_f32(const float* __restrict__ in, float* __restrict__ out,
                       const WarpTask* __restrict__ tasks, int ntasks, const Run2d* __restrict__ runs,
                       const PotConst<float>* __restrict__ consts, unsigned* status) {
    extern __shared__ float4 wring[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = blockIdx.x * kStep2dWarpsPerCta + w;
    if (gw >= ntasks) return;  // whole warp
    const WarpTask task = tasks[gw];
    const Run2d run = runs[task.run];
    const PotConst<float> PC = consts[task.run];
    step2d_strip<VARIANT, POT, STYLE>(in + 4 * run.base, out + 4 * run.base, run.nx, run.ny, task.x0,
                                      task.y_begin, task.y_end, PC, status,
                                      wring + w * (kStep2dStages * 5 * kStep2dWarpRowSites), lane);
}

}  // namespace qlga

