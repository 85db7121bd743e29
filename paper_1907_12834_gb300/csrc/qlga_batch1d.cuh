// qlga_batch1d.cuh -- many independent 1D QLGA lattices of uneven length in one launch per step.
//
// A batch holds nruns periodic 1D lattices back to back; run r occupies its own block of the
// buffer laid out like a single 1D state (5 planes of L_r sites), so plane m of run r starts at
// pair index base_r + m L_r with base_r = 5 sum_{s<r} L_s.  Each run has its own couplings.
//
// One fused step (the state is held pending the kinetic operator, as for a single lattice):
// a CTA of W threads takes one tile of W consecutive sites of one run (the tile table lists
// (run, start) for every tile of every run), stages the tile and its 4-site periodic halo of
// that run in shared memory, applies the nine-point kinetic stencil of the axis (Sec. VII.B)
// and the potential unitary with the run's couplings, and writes the tile: one read and one
// write of the state per step, whatever the mix of lengths.  W is chosen at run time by timing
// the candidates on the live state (see qlga_batch_step).
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"
#include "qlga_step2d.cuh"  // cp.async helpers

namespace qlga {

struct BatchTile {
    int run;
    int start;
};

struct BatchRun {
    int64_t base;  // pair index of plane 0, site 0 of the run
    int L;         // sites of one plane: nx for a 1D run, nx * ny for a 2D run
    int ny;        // 1 for a 1D run
};

template <class T>
struct Pair4 {
    T v[4];  // a.re, a.im, bt.re, bt.im (resident layout)
};

template <class T>
__device__ __forceinline__ Pair4<T> load_raw_pair(const T* X, int64_t pair) {
    Pair4<T> p;
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(X) + pair);
        p.v[0] = v.x; p.v[1] = v.y; p.v[2] = v.z; p.v[3] = v.w;
    } else {
        const double2* q = reinterpret_cast<const double2*>(X) + 2 * pair;
        const double2 u = __ldg(q), w = __ldg(q + 1);
        p.v[0] = u.x; p.v[1] = u.y; p.v[2] = w.x; p.v[3] = w.y;
    }
    return p;
}

template <class T>
__device__ __forceinline__ void store_raw_pair(T* X, int64_t pair, T a0, T a1, T b0, T b1) {
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4*>(X)[pair] = make_float4(a0, a1, b0, b1);
    } else {
        double2* q = reinterpret_cast<double2*>(X) + 2 * pair;
        q[0] = make_double2(a0, a1);
        q[1] = make_double2(b0, b1);
    }
}

// A 1D state held pending K (single lattices and the 1D runs of a batch, both precisions) stores
// each pair as (P, Q) = (a + bt, a - bt), like the fused 2D steps: the nine-point stencil of the
// axis then has 24 nonzero integer taps per level instead of 32 (kStencilPQ, qlga_step2d.cuh).

// Tap K of the kinetic stencil of VARIANT on a neighbour held as (P, Q): (a, bt) accumulators.
template <int VARIANT, int K, class T>
__device__ __forceinline__ void kin_tap_pq(const cpx<T>& P, const cpx<T>& Q, cpx<T>& acc_a, cpx<T>& acc_bt) {
    constexpr KinStencil S = kStencilPQ[VARIANT];
    kin_tap4<S.g[0][0][K], S.g[0][1][K], S.g[1][0][K], S.g[1][1][K]>(P, Q, acc_a, acc_bt);
}

// (P, Q) = (a + i b, a - i b) of a pair (a, b), stored at pair index `pair` of the resident layout
template <class T>
__device__ __forceinline__ void store_raw_pq(T* X, int64_t pair, cpx<T> a, cpx<T> b) {
    store_raw_pair(X, pair, a.re - b.im, a.im + b.re, a.re + b.im, a.im - b.re);
}

// The kinetic operator (nine-point stencil of the axis, Sec. VII.B) at staged column p of src,
// a shared-memory array of 5 planes of `stride` pairs held as (P, Q): the site whose neighbourhood
// is columns p .. p + 8.  Returns (a, b) 16 times the true value (the collides' factors dropped).
template <class T, int VARIANT>
__device__ __forceinline__ void batch_kinetic_at(const Pair4<T>* src, int stride, int p, cpx<T> oa[5],
                                                 cpx<T> ob[5]) {
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        cpx<T> xa = {T(0), T(0)}, xbt = {T(0), T(0)};
        static_for<9>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            const Pair4<T> q = src[m * stride + p + kk];
            kin_tap_pq<VARIANT, kk>(cpx<T>{q.v[0], q.v[1]}, cpx<T>{q.v[2], q.v[3]}, xa, xbt);
        });
        oa[m] = xa;                 // x16, unnormalised
        ob[m] = {xbt.im, -xbt.re};  // b = -i bt
    }
}

// One fused step (POT) or the kinetic operator alone, for the tiles of a batch; with STEPS = 2,
// two fused steps.  The input is held pending K as (P, Q); POT stores (P, Q) again, the kinetic
// operator alone the true state (a, bt).  A CTA of W threads computes W * SPT consecutive sites of one run per pass
// (thread t owns sites t, t + W, ...).  The tile and its periodic halo of 4 * STEPS sites on
// each side are staged in shared memory with 16-byte cp.async copies, all in flight at once.
// STEPS = 2 (temporal blocking): the first step covers the tile and 4 halo sites per side, into
// a second shared buffer; the second step reads that buffer.  The tile is then W * SPT - 8
// sites wide, so both passes fill the threads; the state is read and written once per two
// steps, each site's arithmetic unchanged.
// tiles == nullptr: one 1D lattice of single_L sites with constants single_pc; tile b starts at
// site b * (tile width), and no table is read.
template <class T, int VARIANT, bool POT, int W, int SPT, int STEPS = 1>
__global__ void __launch_bounds__(W) k_batch_step(const T* __restrict__ in, T* __restrict__ out,
                                                   const BatchTile* __restrict__ tiles,
                                                   const BatchRun* __restrict__ runs,
                                                   const PotConst<T>* __restrict__ consts,
                                                   unsigned* status, int single_L,
                                                   PotConst<T> single_pc) {
    static_assert(STEPS == 1 || (STEPS == 2 && POT), "two steps per launch are fused steps");
    constexpr int TW = W * SPT;                  // sites per pass
    constexpr int TOUT = TW - 8 * (STEPS - 1);   // output sites of a tile
    constexpr int H = 4 * STEPS;                 // staged halo per side: TOUT + 2 H = TW + 8
    __shared__ __align__(16) Pair4<T> sm[5][TW + 8];  // 16-byte aligned for cp.async
    __shared__ __align__(16) Pair4<T> mid[5][STEPS == 2 ? TW : 1];
    const bool single = tiles == nullptr;
    const BatchTile tile = single ? BatchTile{0, int(blockIdx.x) * TOUT} : tiles[blockIdx.x];
    const BatchRun run = single ? BatchRun{0, single_L, 1} : runs[tile.run];
    const int L = run.L;
    const int t = threadIdx.x;
    // staged column c holds site start - H + c of the run (periodic)
    auto wrap = [&](int j) {
        if (L >= TW + 8) return j < 0 ? j + L : (j >= L ? j - L : j);  // at most one wrap
        j %= L;
        return j < 0 ? j + L : j;
    };
    auto stage = [&](int c) {
        const int j = wrap(tile.start - H + c);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const T* src = in + 4 * (run.base + int64_t(m) * L + j);
            T* dst = reinterpret_cast<T*>(&sm[m][c]);
#pragma unroll
            for (int q = 0; q < int(sizeof(Pair4<T>)) / 16; ++q) cp_async_16(dst + q * (16 / sizeof(T)), src + q * (16 / sizeof(T)));
        }
    };
#pragma unroll
    for (int k = 0; k < SPT; ++k) stage(4 + t + k * W);
    if (t < 8) stage(t < 4 ? t : TW + t);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const PotConst<T> C = single ? single_pc : consts[tile.run];
    if constexpr (STEPS == 2) {
        // first step on columns 0 .. TW - 1 of mid: sites start - 4 .. start + TOUT + 3
#pragma unroll 1
        for (int k = 0; k < SPT; ++k) {
            const int p = t + k * W;
            cpx<T> oa[5], ob[5];
            batch_kinetic_at<T, VARIANT>(&sm[0][0], TW + 8, p, oa, ob);
            // d takes the degree of psi: one warp-uniform Horner loop (2-3% faster than a per-lane
            // degree for d on the 1D scattering batches and on config 1)
            potential_site<T, false, kZframe64<T>>(oa, ob, C, T(1.0 / 256.0), T(0.5 / 16.0), status);
#pragma unroll
            for (int m = 0; m < 5; ++m)  // held pending K, as (P, Q)
                mid[m][p] = Pair4<T>{{oa[m].re - ob[m].im, oa[m].im + ob[m].re, oa[m].re + ob[m].im, oa[m].im - ob[m].re}};
        }
        __syncthreads();
    }
    const Pair4<T>* src = STEPS == 2 ? &mid[0][0] : &sm[0][0];
    const int stride = STEPS == 2 ? TW : TW + 8;
#pragma unroll 1
    for (int k = 0; k < SPT; ++k) {
        const int tt = t + k * W;
        // positions past the tile's output (STEPS = 2: the last 8) redo a valid site and store nothing
        const int p = tt < TOUT ? tt : TOUT - 1;
        const int j = tile.start + tt;
        cpx<T> oa[5], ob[5];
        batch_kinetic_at<T, VARIANT>(src, stride, p, oa, ob);
        if (POT) {
            // all lanes take part (the Taylor degree is a warp maximum); lanes past the run's end
            // work on a copy of a valid site and store nothing
            potential_site<T, false, kZframe64<T>>(oa, ob, C, T(1.0 / 256.0), T(0.5 / 16.0), status);
        } else {
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                oa[m] = T(1.0 / 16.0) * oa[m];
                ob[m] = T(1.0 / 16.0) * ob[m];
            }
        }
        if (tt < TOUT && j < L) {
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                if (POT)  // held pending K again, as (P, Q)
                    store_raw_pq(out, run.base + int64_t(m) * L + j, oa[m], ob[m]);
                else  // the true state, (a, bt)
                    store_raw_pair(out, run.base + int64_t(m) * L + j, oa[m].re, oa[m].im, -ob[m].im, ob[m].re);
            }
        }
    }
}

}  // namespace qlga
