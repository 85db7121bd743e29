// qlga_interleave.cuh -- fused interleaved QLGA step (arXiv:1907.12834, Sec. VII.B).
//
// The interleaved step applies a fraction U^(1/(4 ndim)) of the potential unitary, re-evaluated
// from the current state, before every kinetic block:
//   for each axis (x, then y):  for c in (2, 2, 1, 1):  psi <- I'_c U^(1/(4 ndim)) psi
// (block order and qubit numbering as in the plain step).  Each block couples a site to its two
// neighbours along the axis, and U is site-local, so one axis is a chain of four (U, block)
// stages with a dependency cone of +-4 sites.  Two kernels do one axis each in a single pass over
// the state:
//
//   k_interleave_x: a CTA of 128 threads owns a tile of up to 120 consecutive sites of one row
//     plus 4 halo sites on each side (periodic); every thread holds one site's 10 amplitudes in
//     registers.  Per stage: U on the site, then the block, whose two streams exchange the shifted
//     qubit with the neighbouring thread through shared memory.  The valid part of the tile
//     shrinks by one site per side per stage; after four stages the 120 interior sites are done.
//   k_interleave_y: a thread owns one column of a row chunk and marches down it; the four stages
//     form a register pipeline (as in the fused plain step): after each input row, U acts on the
//     row leaving stage k and the streaming block k consumes it, so stage k lags by k rows.  The
//     first 8 rows of a chunk only fill the pipeline.
//
// The kinetic arithmetic is unnormalised in the (a, bt = i b) basis: every block multiplies the
// true state by a factor of modulus 2 (2i for K1, 2 for K2).  U is invariant under a global
// factor of modulus 1 and is handed the modulus (inv_sigma2 = 1/4, output scale 1/2), so after
// each U the state carries a pure phase; the phases of the four blocks of one axis multiply to 1
// and each pass ends with the exact factor 2, removed before the store.  Each pass reads and writes
// true states, in the resident layout.
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"

namespace qlga {

constexpr int kIlvXThreads = 128;
constexpr int kIlvXHalo = 4;
constexpr int kIlvXTile = kIlvXThreads - 2 * kIlvXHalo;  // 120 output sites per tile
constexpr int kIlvYThreads = 64;

// Block qubit of stage k: qubit 2 (bt, index 1) twice, then qubit 1 (a, index 0) twice.
__device__ __forceinline__ int ilv_qubit(int k) { return k < 2 ? 1 : 0; }

// Unnormalised collides in the (a, bt) basis: FIRST = 0 is [[1, 1], [-1, 1]] (K1's C, and both
// variants' C'), FIRST = 1 is [[1, -1], [1, 1]] (K2's C).
template <class T, int FIRST>
__device__ __forceinline__ void ilv_collide(cpx<T>& a, cpx<T>& bt) {
    const cpx<T> x = a, y = bt;
    if (FIRST == 0) {
        a = x + y;
        bt = y - x;
    } else {
        a = x - y;
        bt = x + y;
    }
}

// U on one site held as (a, bt): converts to (a, b), applies the potential, converts back.
template <class T>
__device__ __forceinline__ void ilv_potential(cpx<T> a[5], cpx<T> bt[5], const PotConst<T>& PC, T inv_sigma2,
                                              T out_scale, unsigned* status) {
    cpx<T> b[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) b[m] = {bt[m].im, -bt[m].re};  // b = -i bt
    potential_site<T, sizeof(T) == 4>(a, b, PC, inv_sigma2, out_scale, status);
#pragma unroll
    for (int m = 0; m < 5; ++m) bt[m] = {-b[m].im, b[m].re};  // bt = i b
}

template <class T>
__device__ __forceinline__ void ilv_load(const T* X, int64_t nsites, int64_t site, cpx<T> a[5], cpx<T> bt[5]) {
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        if constexpr (sizeof(T) == 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(X) + m * nsites + site);
            a[m] = {v.x, v.y};
            bt[m] = {v.z, v.w};
        } else {
            const double2* p = reinterpret_cast<const double2*>(X) + 2 * (m * nsites + site);
            const double2 u = __ldg(p), w = __ldg(p + 1);
            a[m] = {u.x, u.y};
            bt[m] = {w.x, w.y};
        }
    }
}

template <class T>
__device__ __forceinline__ void ilv_store(T* X, int64_t nsites, int64_t site, const cpx<T> a[5],
                                          const cpx<T> bt[5], T s) {
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        if constexpr (sizeof(T) == 4) {
            reinterpret_cast<float4*>(X)[m * nsites + site] =
                make_float4(s * a[m].re, s * a[m].im, s * bt[m].re, s * bt[m].im);
        } else {
            double2* p = reinterpret_cast<double2*>(X) + 2 * (m * nsites + site);
            p[0] = make_double2(s * a[m].re, s * a[m].im);
            p[1] = make_double2(s * bt[m].re, s * bt[m].im);
        }
    }
}

// ------------------------------------------------------------------ x axis

template <class T, int VARIANT>
__global__ void __launch_bounds__(kIlvXThreads) k_interleave_x(const T* __restrict__ in, T* __restrict__ out,
                                                               int64_t nx, int64_t ny, PotConst<T> PC,
                                                               unsigned* status) {
    __shared__ cpx<T> s1[5][kIlvXThreads];
    __shared__ cpx<T> s2[5][kIlvXThreads];
    const int t = threadIdx.x;
    const int64_t tiles_per_row = (nx + kIlvXTile - 1) / kIlvXTile;
    const int64_t ntiles = tiles_per_row * ny;
    const int64_t nsites = nx * ny;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t y = tile / tiles_per_row;
        const int64_t x0 = (tile - y * tiles_per_row) * kIlvXTile;
        const int w = int(nx - x0 < kIlvXTile ? nx - x0 : kIlvXTile);  // output sites of this tile
        // thread t holds column x0 - 4 + t (periodic); the tile needs t in [0, w + 8)
        int64_t col = (x0 - kIlvXHalo + t) % nx;
        col = col < 0 ? col + nx : col;
        const int64_t site = y * nx + col;
        cpx<T> a[5], bt[5];
        ilv_load(in, nsites, site, a, bt);
        if (t >= w + 2 * kIlvXHalo) {
#pragma unroll
            for (int m = 0; m < 5; ++m) a[m] = bt[m] = {T(0), T(0)};
        }
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            // U^(delta) on the site (the state carries a factor of modulus 2 after a block)
            ilv_potential(a, bt, PC, k == 0 ? T(1) : T(0.25), k == 0 ? T(0.5) : T(0.25), status);
            const int c = ilv_qubit(k);
            // first collide, then S^T_c: qubit c of site j takes qubit c of site j + 1
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                if (VARIANT == 0) ilv_collide<T, 0>(a[m], bt[m]);
                else ilv_collide<T, 1>(a[m], bt[m]);
                s1[m][t] = c == 0 ? a[m] : bt[m];
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const cpx<T> z = t + 1 < kIlvXThreads ? s1[m][t + 1] : cpx<T>{T(0), T(0)};
                if (c == 0) a[m] = z;
                else bt[m] = z;
                ilv_collide<T, 0>(a[m], bt[m]);  // C'
                s2[m][t] = c == 0 ? a[m] : bt[m];
            }
            __syncthreads();
            // S_c: qubit c of site j takes qubit c of site j - 1
            const bool valid = t >= k + 1 && t < w + 2 * kIlvXHalo - k - 1;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const cpx<T> z = t >= 1 ? s2[m][t - 1] : cpx<T>{T(0), T(0)};
                if (c == 0) a[m] = z;
                else bt[m] = z;
                if (!valid) a[m] = bt[m] = {T(0), T(0)};
            }
        }
        if (t >= kIlvXHalo && t < kIlvXHalo + w) ilv_store(out, nsites, site, a, bt, T(0.5));
        __syncthreads();  // the next tile reuses s1 / s2
    }
}

// ------------------------------------------------------------------ y axis

// One streaming block along y for one level (input row n -> output row n - 1, in place); the
// state keeps the unshifted qubit after the first collide (yo) and the shifted qubit after the
// second (wc) from the previous row.  C = 1 shifts bt, C = 0 shifts a.  The new yo is formed from
// the inputs only after the old one has been used, so that the loop-carried value can keep its
// register from row to row.
template <class T, int FIRST>
__device__ __forceinline__ void ilv_stream(int c, cpx<T>& a, cpx<T>& bt, cpx<T>& yo, cpx<T>& wc) {
    const cpx<T> ia = a, ibt = bt;
    if (c == 1) {
        const cpx<T> ybt = FIRST == 0 ? ibt - ia : ia + ibt;
        const cpx<T> wa = yo + ybt, wbt = ybt - yo;  // second collide of (yo, ybt)
        yo = FIRST == 0 ? ia + ibt : ia - ibt;
        a = wa;
        bt = wc;
        wc = wbt;
    } else {
        const cpx<T> ya = FIRST == 0 ? ia + ibt : ia - ibt;
        const cpx<T> wa = ya + yo, wbt = yo - ya;  // second collide of (ya, yo)
        yo = FIRST == 0 ? ibt - ia : ia + ibt;
        a = wc;
        bt = wbt;
        wc = wa;
    }
}

template <class T, int VARIANT>
// FP32: 8 resident CTAs per SM (128 registers, a few spilled) beat 6 at 168 registers by 8%;
// FP64 keeps the register budget.
__global__ void __launch_bounds__(kIlvYThreads, sizeof(T) == 4 ? 8 : 1) k_interleave_y(const T* __restrict__ in, T* __restrict__ out,
                                                               int64_t nx, int64_t ny, int chunks,
                                                               PotConst<T> PC, unsigned* status) {
    const int64_t strips = (nx + kIlvYThreads - 1) / kIlvYThreads;
    const int64_t nsites = nx * ny;
    const int64_t strip = blockIdx.x % strips;
    const int64_t chunk = blockIdx.x / strips;
    const int64_t xcol = strip * kIlvYThreads + threadIdx.x;
    const bool active = xcol < nx;
    const int64_t x = active ? xcol : nx - 1;
    const int64_t y_begin = (chunk * ny) / chunks, y_end = ((chunk + 1) * ny) / chunks;
    const int64_t nrows = (y_end - y_begin) + 8;
    cpx<T> yo[4][5], wc[4][5];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m < 5; ++m) yo[k][m] = wc[k][m] = {T(0), T(0)};
#pragma unroll 1
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t yy = y_begin - 4 + r;
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        cpx<T> a[5], bt[5];
        ilv_load(in, nsites, yy * nx + x, a, bt);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ilv_potential(a, bt, PC, k == 0 ? T(1) : T(0.25), k == 0 ? T(0.5) : T(0.25), status);
            const int c = ilv_qubit(k);
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                if (VARIANT == 0) ilv_stream<T, 0>(c, a[m], bt[m], yo[k][m], wc[k][m]);
                else ilv_stream<T, 1>(c, a[m], bt[m], yo[k][m], wc[k][m]);
            }
        }
        if (r >= 8 && active) ilv_store(out, nsites, (y_begin + r - 8) * nx + x, a, bt, T(0.5));
    }
}

}  // namespace qlga
