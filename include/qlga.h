/*
 * qlga.h — C ABI of the spin-2 BEC quantum lattice gas algorithm (QLGA) library.
 *
 * The library advances the 10-qubit-per-site QLGA state of a spin-2 Bose-Einstein
 * condensate (Taylor, Smith & Yepez, arXiv:1907.12834) on one GPU.  One time step is
 *
 *     psi(t + tau) = (I'_1 I'_1 I'_2 I'_2 U) psi(t)            (Sec. VII.B, operator
 *                                                               product of the plain step)
 *
 * with the self-interaction unitary U = exp(-i delta V(psi)) applied first, then the kinetic
 * blocks I'_c = S_c C S^T_c C along x (and then along y in 2D).
 *
 * ---------------------------------------------------------------------------------------
 * State layout ("qubit-pair planes").  Every state buffer, on the host or on the device,
 * holds 5 planes, one per Zeeman level m = +2, +1, 0, -1, -2 (in that order).  A plane
 * holds ny*nx sites, x fastest.  A site holds the two qubit amplitudes of that level
 * (Sec. III.B, Eq. full_state: two qubits per m_f) as four reals:
 *
 *     a.re, a.im, b.re, b.im        (a = first qubit of the pair, b = second)
 *
 * so element (m, y, x, q, c) sits at offset (((m*ny + y)*nx + x)*2 + q)*2 + c.  The reals
 * are float for precision 32 and double for precision 64.  The boson field of level m is
 * psi_m = a_m + b_m; a boson field psi loaded with qlga_load_boson() is split as
 * a = b = eps*psi/2 (Sec. VII.A, Eq. eomscaling: psi_lattice = sqrt(gamma) psi, gamma = eps^2).
 *
 * Lattice units: x = eps*j, t = eps^2*n.  Periodic boundaries on every axis.
 *
 * Ownership.  qlga_create() allocates the device state and work buffers with cudaMalloc
 * and qlga_destroy() frees them.  qlga_create_external() uses caller-owned device buffers
 * instead; the caller keeps them alive until qlga_destroy().  Host buffers always belong to
 * the caller.
 *
 * Streams and threading.  Every call that launches work enqueues it on the handle's CUDA
 * stream (the one passed at creation; NULL = the legacy default stream).  qlga_step() returns
 * before the work finishes; qlga_observables(), qlga_get_state() to the host and
 * qlga_synchronize() wait for the stream.  A handle must not be used from two host threads at
 * once.
 *
 * Errors.  Every call returns a qlga_status and never aborts the process.  After an error,
 * qlga_last_error() returns a one-line description (per host thread).
 * ---------------------------------------------------------------------------------------
 */
#ifndef QLGA_H
#define QLGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qlga_status {
    QLGA_OK = 0,
    QLGA_ERR_INVALID_ARG = 1,   /* a NULL pointer, a bad size, a bad enum value              */
    QLGA_ERR_OOM = 2,           /* cudaMalloc failed                                          */
    QLGA_ERR_CUDA = 3,          /* a CUDA runtime call or a kernel launch failed              */
    QLGA_ERR_TIMEOUT = 4,       /* reserved for a bounded device wait that gives up; no kernel of this
                                   library waits on another CTA or on the host, so none returns it */
    QLGA_ERR_NOT_FINITE = 5,    /* the state holds NaN or Inf                                 */
    QLGA_ERR_UNSUPPORTED = 6    /* a valid configuration that this build does not implement   */
} qlga_status;

/* Where a buffer passed to load/get lives. */
enum { QLGA_HOST = 0, QLGA_DEVICE = 1 };

/* Collide reading (Sec. VII.B: the collide matrix itself is given in a cited work that the
 * paper does not reproduce).
 *   QLGA_KINETIC_K1: I'_c = S_c C S^T_c C with C = 1/2 [[1-i, 1+i], [1+i, 1-i]] (default).
 *   QLGA_KINETIC_K2: I'_c = S_c C^dagger S^T_c C with C = 1/2 [[1+i, 1-i], [1-i, 1+i]].   */
enum { QLGA_KINETIC_K1 = 0, QLGA_KINETIC_K2 = 1 };

typedef struct qlga_config {
    int32_t ndim;            /* 1 or 2                                                       */
    int32_t precision;       /* 32 (float) or 64 (double)                                    */
    int64_t nx;              /* sites along x, >= 8                                          */
    int64_t ny;              /* sites along y, >= 8 for ndim 2; must be 1 for ndim 1         */
    double g0, g1, g2;       /* density, spin-density and singlet couplings (Sec. II, the
                                spin-2 interaction Hamiltonian Eq. hamspin2)                 */
    double epsilon;          /* lattice scaling of Sec. VII.A; used only by qlga_load_boson  */
    int32_t interleave;      /* 0: plain step (Sec. VII.B).  1: interleaved step, U^(1/4)
                                (1D) or U^(1/8) (2D) before every kinetic block             */
    int32_t kinetic_variant; /* QLGA_KINETIC_K1 or QLGA_KINETIC_K2                          */
} qlga_config;

/* Global observables of the boson field psi = a + b at the current time (FP64 sums).
 * Sec. III.B characteristics (Eq. cmap), Sec. IV.B discrete energy (Eq. disecrete_energy). */
typedef struct qlga_obs {
    double norm_qubit;        /* sum |a|^2 + |b|^2 over sites and levels (exactly conserved) */
    double norm_boson;        /* sum |psi|^2                                                 */
    double pop[5];            /* qubit population of m = +2..-2: sum |a_m|^2 + |b_m|^2       */
    double magnetisation;     /* sum_m m * pop[m]                                           */
    double energy;            /* sum over sites of sum_axis sum_m |psi_m(j+1) - psi_m(j)|^2
                                 + g0/2 rho^2 + g1/2 |F|^2 + g2/10 |psi^T J psi|^2           */
    double singlet_re;        /* sum psi^T J psi / sqrt(5), (J psi)_m = (-1)^m psi_{-m}       */
    double singlet_im;
    double singlet_fraction;  /* sum |psi^T J psi|^2 / sum rho^2                             */
    double overlap_re;        /* <psi(t) | ref> when a reference state was given, else 0     */
    double overlap_im;
    int64_t step;             /* time steps taken since the last load                        */
} qlga_obs;

typedef struct qlga_handle qlga_handle;

/* Bytes of one state buffer for this configuration (5 * 4 * nx * ny reals). */
qlga_status qlga_state_bytes(const qlga_config* cfg, size_t* bytes);

/* Bytes of device work memory that qlga_create_external() needs beside the two state
 * buffers (one more state buffer plus the reduction partials). */
qlga_status qlga_workspace_bytes(const qlga_config* cfg, size_t* bytes);

/* Validate cfg, allocate the state (two ping-pong buffers) and the workspace on the current
 * device, and bind the handle to `stream` (a cudaStream_t, may be NULL).  The state starts
 * at zero.  INVALID_ARG for a bad config, OOM when cudaMalloc fails. */
qlga_status qlga_create(const qlga_config* cfg, void* stream, qlga_handle** out);

/* Same as qlga_create() but on caller-owned device memory: state0 and state1 each of
 * qlga_state_bytes(), workspace of at least qlga_workspace_bytes(); all 256-byte aligned.
 * Nothing is allocated on the device. */
qlga_status qlga_create_external(const qlga_config* cfg, void* stream, void* state0,
                                 void* state1, void* workspace, size_t workspace_bytes,
                                 qlga_handle** out);

/* Load a full 10-amplitude state (layout above, the handle's precision) from host or device
 * memory.  Resets the step counter.  A host load is a synchronous copy. */
qlga_status qlga_load_state(qlga_handle* h, const void* src, int where);

/* Load a physical boson field psi (complex, [5][ny][nx], re/im interleaved, the handle's
 * precision): a = b = epsilon * psi / 2 (Sec. VII.A scaling). */
qlga_status qlga_load_boson(qlga_handle* h, const void* psi5, int where);

/* Copy the current state (layout above) to host or device memory.  A host copy waits. */
qlga_status qlga_get_state(qlga_handle* h, void* dst, int where);

/* Advance n >= 0 time steps (asynchronous on the handle's stream). */
qlga_status qlga_step(qlga_handle* h, int64_t n);

/* Apply only the self-interaction unitary U = exp(-i delta V(psi)) to every site, or only
 * the kinetic operator (all axes), to the current state.  Stage-wise entry points for
 * checking the two halves of the step separately (Sec. VII.B). */
qlga_status qlga_apply_potential(qlga_handle* h, double delta);
qlga_status qlga_apply_kinetic(qlga_handle* h);

/* Global observables of the current state; waits for the stream.  `ref_state_device` may
 * be NULL; otherwise it is a device state of the same shape and precision and the overlap
 * <psi(t) | psi_ref> of the boson fields is filled in (the discrete energy of Sec. IV.B). */
qlga_status qlga_observables(qlga_handle* h, const void* ref_state_device, qlga_obs* out);

/* ---------------------------------------------------------------------------------------
 * Slab decomposition (Sec. VII.C, "Speed, size and scalability": the lattice is split over
 * several GPUs).  A 2D lattice of nx x ny sites is cut along y into slabs; each slab is an
 * ordinary handle whose lattice holds the slab's rows plus a halo of H >= 5 rows on each side
 * (its own periodic wrap in y only ever touches the halo).  One step moves a site's
 * dependency cone at most 4 rows along y (the four kinetic blocks of the axis), so if the halo
 * rows hold the neighbouring slabs' rows before every qlga_step(h, 1), the slab's own rows come
 * out exactly as in the whole lattice; halo rows hold stale values after a step until the next
 * exchange.  The fifth halo row serves the forward difference of the energy at the slab's last
 * row.  A read-out (qlga_get_state, qlga_observable_sums) also needs fresh halo rows.
 * --------------------------------------------------------------------------------------- */
enum { QLGA_ROWS_OUT = 0, QLGA_ROWS_IN = 1 };

/* Copy rows [y0, y0 + nrows) of all 5 planes of the handle's current state buffer, as held
 * (the library's own representation, opaque to the caller), to (QLGA_ROWS_OUT) or from
 * (QLGA_ROWS_IN) `buf`: device memory of 5 * nrows * nx * 16 bytes (FP32) or 32 (FP64), laid
 * out [plane][row][x], owned by the caller.  Enqueued on the handle's stream (one
 * cudaMemcpy2DAsync).  The rows move between handles of the same nx and precision that have
 * taken the same steps, e.g. through NCCL send / recv between ranks.  INVALID_ARG for rows
 * outside the lattice or a bad direction. */
qlga_status qlga_copy_rows(qlga_handle* h, int64_t y0, int64_t nrows, void* buf, int direction);

/* Copy rows [ysrc, ysrc + nrows) of src's current state buffer into rows [ydst, ...) of
 * dst's: two handles of the same nx, precision and dimension that have taken the same steps,
 * on one device or on two devices with peer access.  The copy runs on dst's stream after the
 * work queued on src's stream, and src's stream waits for it.  INVALID_ARG for mismatched
 * handles, rows outside a lattice or overlapping rows of one handle. */
qlga_status qlga_exchange_rows(qlga_handle* src, int64_t ysrc, qlga_handle* dst, int64_t ydst,
                               int64_t nrows);

/* The 14 FP64 sums behind qlga_obs over the rows [y0, y1) of the current true state (the
 * forward difference of row y1 - 1 reads row y1, or row 0 when y1 == ny), written to sums[14]
 * (host memory): qubit norm, boson norm, the 5 populations, energy, singlet amplitude (re,
 * im), sum |psi^T J psi|^2, sum rho^2 and the overlap with `ref_state_device` (re, im; 0 when
 * it is NULL).  Sums of disjoint row ranges add up (an all-reduce over slabs); waits for the
 * stream.  Sec. III.B Eq. cmap, Sec. IV.B Eq. disecrete_energy. */
qlga_status qlga_observable_sums(qlga_handle* h, int64_t y0, int64_t y1, const void* ref_state_device,
                                 double* sums);

/* qlga_obs from the 14 sums of qlga_observable_sums (host only): magnetisation and singlet
 * fraction are formed from the sums.  NOT_FINITE when the norm or the energy is not finite. */
qlga_status qlga_obs_from_sums(const double* sums, int64_t step, qlga_obs* out);

/* Objectives of a state that gradients are taken of, with their cotangent (Sec. III.B Eq. cmap:
 * the populations and the singlet pair amplitude psi^T J psi; the energy is the functional
 * whose variation is the right-hand side of Eq. eomspin2, forward differences for the
 * gradient term, as in qlga_obs):
 *   values[0] = P = sum |a_l|^2 + |b_l|^2 of level `level` (0..4 for m = +2..-2),
 *   values[1] = S = sum |psi^T J psi|^2 / sum rho^2 (the singlet fraction),
 *   values[2] = E = sum_sites [sum_axis sum_m |psi_m(j+1) - psi_m(j)|^2 + g0/2 rho^2
 *                              + g1/2 |F|^2 + g2/10 |psi^T J psi|^2]   with the couplings g[3].
 * `x_device` is a state of the handle's shape and precision in the layout above (device
 * memory, caller-owned, not the handle's own buffers).  With `cot_device` (same shape, layout
 * and precision, device memory) the call also writes the cotangent of L = weights[0] P +
 * weights[1] S + weights[2] E: dL/d(each real of the state), i.e. dL/dRe z + i dL/dIm z per
 * amplitude; with `dg` (3 host doubles) it writes L's own dependence on the couplings, dL/dg0 =
 * weights[2] sum rho^2 / 2, dL/dg1 = weights[2] sum |F|^2 / 2, dL/dg2 = weights[2] sum
 * |psi^T J psi|^2 / 10.  Sums in FP64 (compensated per thread for FP32 states); uses the
 * handle's work memory and stream and waits for it.  INVALID_ARG for a bad level, missing
 * weights, or non-finite couplings; NOT_FINITE for a state holding NaN or Inf. */
qlga_status qlga_objective(qlga_handle* h, const void* x_device, int32_t level, const double* g,
                           const double* weights, double* values, double* dg, void* cot_device);

/* Per-site diagnostic fields of the current state (Sec. III.B Eq. cmap and Eq. colormap,
 * Sec. VI.B Eqs. velocity / pointwise_vorticity), written to `dst` as 11 planes of ny*nx
 * values in the handle's precision, x fastest:
 *   0 F_par = sum_m m |psi_m|^2          1 F_perp = |psi^dagger (f_x + i f_y) psi|
 *   2 |A00| = |psi^T J psi| / sqrt(5)   3..5 (r, g, b) = (|F_par|, F_perp, |A00|) / their norm
 *                                           (0 where all three vanish)
 *   6..10 vorticity of level m = +2..-2: phase S = arg psi_m, v = wrapped central differences
 *         of S / 2, vorticity = central-difference curl of v (0 in 1D).  The unwrapped parts of
 *         the four differences cancel, so the value is pi/2 times an integer, the sum of their
 *         wrap counts; the counts are those of the FP64 phases in both precisions (phases near a
 *         wrap decision are taken again in FP64).
 * `where` is QLGA_HOST or QLGA_DEVICE; a host copy waits for the stream. */
qlga_status qlga_fields(qlga_handle* h, void* dst, int where);

/* Observables of a caller-provided device state without allocating any device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot allocate:
 * code whose device memory is owned by its own allocator or by a fixed memory plan (a caching
 * allocator that has reserved the pool, a service with a preset budget), where a cudaMalloc
 * issued by the library could fail or fragment that pool, and time-critical loops that must not
 * stall on cudaMalloc / cudaFree, which can synchronise the device.  It computes the same sums
 * as qlga_observables() (step is reported as 0) for `state_device`, a state in the layout above
 * in the precision of `cfg`, with `ref_state_device` optional as there; `stream` is a
 * cudaStream_t (NULL = legacy default stream) and the call waits for it.  No handle is needed.
 *
 * Scratch: the block partial sums live in one file-scope __device__ array of 1216 partial rows
 * of 14 doubles plus the 14 results (136,304 bytes), which every GPU that loads the library
 * holds until the process exits.  The reduction is a grid-stride loop over at most 1216 blocks,
 * one partial row each, so every configuration that qlga_state_bytes() accepts fits; a
 * configuration it rejects is rejected here with QLGA_ERR_INVALID_ARG.  Nothing is allocated: no
 * cudaMalloc, cudaFree or allocating library routine is called.
 *
 * Each call, on the current device, looks up the device address of the array with
 * cudaGetSymbolAddress (it allocates nothing, and a fresh lookup stays valid after a
 * cudaDeviceReset), launches the reduction on `stream`, copies the 14 results to `out` and waits
 * for `stream` to finish.  All calls on a device share the one array, which keeps the last
 * call's contents; each call overwrites every partial row it reads, so nothing needs clearing,
 * but calls whose work overlaps on the GPU (different streams or host threads) race on the
 * array and must be serialised by the caller. */
qlga_status qlga_observables_noalloc(const qlga_config* cfg, const void* state_device,
                                     const void* ref_state_device, void* stream, qlga_obs* out);

/* Steps per CUDA graph replay.  On lattices of at most 2^18 sites the step is bound by launch
 * latency, so qlga_step() replays runs of `steps` fused steps (default 32) from a graph captured
 * on first use (the same kernels with the same arguments; results are identical).  steps must be
 * even, 0..4096; 0 turns graphs off.  Larger lattices start with 0. */
qlga_status qlga_set_graph_steps(qlga_handle* h, int32_t steps);

/* Which kernel runs a step on a 2D lattice.  Sec. VII.B's step is the same either way; the two
 * forms differ only in how the passes are grouped, and their results agree to rounding.
 *   QLGA_STEP2D_AUTO      (default) the fused single-pass kernel when nx is a multiple of 32 and,
 *                         in FP64, a cost estimate favours it (on small FP64 lattices each row
 *                         chunk's warm-up rows outweigh the saved pass);
 *   QLGA_STEP2D_FUSED     always the fused kernel (warp strips of 32 columns: nx % 32 == 0);
 *   QLGA_STEP2D_TWO_PASS  always two passes: x, then y with the potential.
 * Errors: QLGA_ERR_INVALID_ARG for an unknown mode, QLGA_ERR_UNSUPPORTED for QLGA_STEP2D_FUSED
 * on a 1D lattice or nx not a multiple of 32.  Changing the mode waits for the handle's stream
 * and drops captured step graphs.  qlga_get_step2d_kernel() reports the form the next step uses
 * (QLGA_STEP2D_FUSED or QLGA_STEP2D_TWO_PASS; 0 on a 1D lattice). */
#define QLGA_STEP2D_AUTO 0
#define QLGA_STEP2D_FUSED 1
#define QLGA_STEP2D_TWO_PASS 2
qlga_status qlga_set_step2d_mode(qlga_handle* h, int32_t mode);
qlga_status qlga_get_step2d_kernel(qlga_handle* h, int32_t* kernel);

/* Launch shape of a 1D lattice's steps: the tiled kernel the batches use (tiles computed from the
 * block index), or the lane-parallel kernel for small lattices whose one-site-per-thread launches
 * leave most of the GPU idle: shape (5, 0, 1), a site's five levels on five lanes, six sites per
 * warp; or (10, 0, 1), the psi and d = a - b recursions of U on separate lanes, three sites per
 * warp.  The first fused step times the candidates on the live state and keeps the fastest per
 * step: a one-step shape, in FP32 plain steps a two-step shape (temporal blocking, see the
 * batches; qlga_step then takes fused steps two per launch), or, in FP64, a lane-parallel kernel
 * (in FP32 it can be forced: its Taylor degree, a maximum over 3 or 6 sites instead of 32,
 * truncates closer to the tolerance).
 * qlga_set_1d_shape forces a shape (the list of qlga_batch_set_shape, (5, 0, 1), (10, 0, 1), or
 * the (0, 0, 0) reset); qlga_get_1d_shape reports the one fused steps use (zeros before tuning).  Setting waits for the
 * handle's stream and drops captured step graphs.  Errors: QLGA_ERR_UNSUPPORTED on a 2D lattice,
 * or two steps per launch in FP64 or with interleave; QLGA_ERR_INVALID_ARG for another shape. */
qlga_status qlga_set_1d_shape(qlga_handle* h, int32_t threads, int32_t sites_per_thread, int32_t steps);
qlga_status qlga_get_1d_shape(qlga_handle* h, int32_t* threads, int32_t* sites_per_thread, int32_t* steps);

/* Number of kernels this handle has launched since creation (a diagnostic for benchmarks). */
qlga_status qlga_launch_count(const qlga_handle* h, int64_t* count);

/* Wait for all work enqueued on the handle's stream. */
qlga_status qlga_synchronize(qlga_handle* h);

/* Free the handle (and the device memory that qlga_create() allocated).  NULL is OK. */
qlga_status qlga_destroy(qlga_handle* h);

/* ---------------------------------------------------------------------------------------
 * Adjoint (reverse mode): gradients of a real loss L of the state after n plain steps
 * x_{k+1} = K U(x_k) x_k (Sec. VII.B), with respect to the initial state x_0 and the couplings
 * (g0, g1, g2) of Eq. hamspin2.
 *
 * Cotangents.  A cotangent buffer has the state layout and precision above and holds
 * dL/d(each real of the state): element (m, y, x, q, c) is dL/d(Re or Im of a or b).  So
 * dL = sum over all elements of cot * dx.  One step pulls a cotangent back as
 * cot_k = (d x_{k+1} / d x_k)^T cot_{k+1}: the adjoint kinetic operator K^dagger (axes and blocks
 * in reverse order, each collide and stream replaced by its adjoint), then the transposed
 * linearisation of U at x_k, which includes the dependence of V on psi = a + b (Frechet
 * derivative of exp(-i delta V), evaluated with the forward step's own Taylor degree).
 *
 * Checkpoints.  qlga_adjoint_forward() keeps the true state every C steps (x_0, x_C, ...) in the
 * workspace; qlga_adjoint_backward() recomputes each segment of C states from its checkpoint
 * (C extra state buffers) and pulls the cotangent back through it.  Checkpoints are held in the
 * handle's precision: a recomputed segment repeats the forward arithmetic of that precision.
 * Workspace: qlga_adjoint_workspace_bytes() bytes of device memory, 256-byte aligned, owned by
 * the caller; about (ceil(n / C) + C + 4) state buffers.  The same workspace must be passed to
 * the forward and the backward call of one run, unchanged in between.
 *
 * The adjoint covers the plain step only: a handle with interleave = 1 gets
 * QLGA_ERR_UNSUPPORTED.  dcoup (host, 3 doubles) receives dL/d(g0, g1, g2) and may be NULL.
 * All three calls enqueue on the handle's stream; backward and step wait for it before
 * returning (they read dcoup back).  A status word set by U (exponent out of range) is reported
 * as QLGA_ERR_NOT_FINITE, as for the forward step. */
qlga_status qlga_adjoint_workspace_bytes(const qlga_config* cfg, int64_t nsteps, int64_t checkpoint_every,
                                         size_t* bytes);

/* Load x0 (device, state layout) into the handle, advance it nsteps plain steps (the handle ends
 * holding x_n, as after qlga_load_state + qlga_step) and store the checkpoints. */
qlga_status qlga_adjoint_forward(qlga_handle* h, const void* x0_device, int64_t nsteps, int64_t checkpoint_every,
                                 void* workspace, size_t workspace_bytes);

/* cot_device (device, cotangent layout): dL/dx_n on entry, dL/dx_0 on exit, using the
 * checkpoints of the preceding qlga_adjoint_forward() with the same nsteps and
 * checkpoint_every.  Does not change the handle's state. */
qlga_status qlga_adjoint_backward(qlga_handle* h, int64_t nsteps, int64_t checkpoint_every, void* workspace,
                                  size_t workspace_bytes, void* cot_device, double* dcoup);

/* qlga_adjoint_forward followed by qlga_adjoint_backward. */
qlga_status qlga_adjoint_run(qlga_handle* h, const void* x0_device, int64_t nsteps, int64_t checkpoint_every,
                             void* workspace, size_t workspace_bytes, void* cot_device, double* dcoup);

/* One step pulled back at the state x_device (device, state layout): cot_device holds
 * dL/dx_{k+1} on entry and dL/dx_k on exit.  Workspace as for nsteps = 1,
 * checkpoint_every = 1.  Does not change the handle's state. */
qlga_status qlga_adjoint_step(qlga_handle* h, const void* x_device, void* cot_device, void* workspace,
                              size_t workspace_bytes, double* dcoup);

/* ---------------------------------------------------------------------------------------
 * Batches: many independent periodic lattices of uneven size, 1D and 2D, each with its own
 * couplings, advanced together.  The state buffer of a batch is the concatenation of the runs'
 * states, each in the layout above (run r starts at element 20 * sum_{s<r} nx_s ny_s).  Steps are
 * the plain step.  1D runs go through a tiled kernel (Sec. VII.B's step on each tile and its
 * periodic halo); the first qlga_batch_step() times its candidate launch shapes on the live state
 * (writing only work space) and keeps the fastest: tiles of 32 / 64 / 128 / 256 sites at 1 / 2 / 4
 * sites per thread, one step per launch, and -- FP32 batches of 1D runs only -- two steps per
 * launch on tiles of 120 / 248 sites (temporal blocking: the tile and an 8-site halo are read
 * once, the first step's result stays in shared memory; each site's arithmetic is unchanged), if
 * that is faster per step.  2D runs (FP32; nx a multiple of 32) go through the fused warp-strip
 * kernel of the single 2D lattice, its warps reading their run, strip and row range from a task
 * table, in one more launch per step.  On a non-default stream, runs of steps (two launches) are
 * replayed from a CUDA graph captured once.
 * --------------------------------------------------------------------------------------- */
typedef struct qlga_batch_config {
    int32_t precision;       /* 32 or 64 (64: 1D runs only) */
    int32_t nruns;           /* >= 1 */
    const int64_t* lengths;  /* host array [nruns]: nx of each run; a 1D run has 8 <= nx <= 2^30 */
    const double* couplings; /* host array [nruns][3]: g0, g1, g2 of each run */
    double epsilon;          /* lattice scaling (informational for batches) */
    int32_t kinetic_variant; /* QLGA_KINETIC_K1 or QLGA_KINETIC_K2 */
    int32_t use_graph;       /* 1: replay steps from a captured CUDA graph where possible */
    const int64_t* heights;  /* host array [nruns]: ny of each run (1: a 1D run; a 2D run needs
                                ny >= 8, nx a multiple of 32, nx * ny <= 2^30), or NULL: all 1D */
} qlga_batch_config;

typedef struct qlga_batch qlga_batch;

/* Bytes of the batch state (20 reals per site summed over runs). */
qlga_status qlga_batch_state_bytes(const qlga_batch_config* cfg, size_t* bytes);

/* Allocate a batch on the current device (two state buffers, work space, per-run tables). */
qlga_status qlga_batch_create(const qlga_batch_config* cfg, void* stream, qlga_batch** out);

/* Load / read the concatenated state (host or device memory; host calls wait). */
qlga_status qlga_batch_load_state(qlga_batch* b, const void* src, int where);
qlga_status qlga_batch_get_state(qlga_batch* b, void* dst, int where);

/* Advance every run n >= 0 steps (asynchronous). */
qlga_status qlga_batch_step(qlga_batch* b, int64_t n);

/* Observables of every run: out is a host array of nruns qlga_obs (FP64 sums); waits. */
qlga_status qlga_batch_observables(qlga_batch* b, qlga_obs* out);

/* Launch shape of the 1D runs' steps (0 before the first step): tile width in sites, sites per
 * thread and fused steps per launch (1, or 2 with temporal blocking; the CTA has
 * (tile_width + 8 (steps - 1)) / sites_per_thread threads); kernels launched, and the number of
 * steps taken through graph replays.  Any pointer may be NULL. */
qlga_status qlga_batch_info(const qlga_batch* b, int32_t* tile_width, int32_t* sites_per_thread,
                            int64_t* launches, int64_t* graph_steps, int32_t* steps_per_launch);

/* Force the launch shape of the 1D runs instead of timing the candidates: (threads per CTA,
 * sites per thread, steps per launch) is one of (32, 1, 1), (64, 1, 1), (128, 1, 1), (256, 1, 1),
 * (64, 2, 1), (128, 2, 1), (64, 4, 1), (64, 4, 2), (128, 2, 2), (64, 2, 2), (256, 1, 2); with two
 * steps per launch, single steps (an odd count) take the same threads and sites per thread.
 * (0, 0, 0) returns to timing the candidates at the next step.  Results agree with every shape
 * to rounding (the Taylor degree of U is a warp maximum).  Waits for the batch's stream and drops
 * its captured graph.  Errors: QLGA_ERR_INVALID_ARG for another shape, QLGA_ERR_UNSUPPORTED for
 * two steps per launch in an FP64 batch or one with 2D runs. */
qlga_status qlga_batch_set_shape(qlga_batch* b, int32_t threads, int32_t sites_per_thread, int32_t steps);

qlga_status qlga_batch_destroy(qlga_batch* b);

/* Static description of a status code. */
const char* qlga_status_string(qlga_status s);

/* One-line description of the last error on this host thread ("" when none). */
const char* qlga_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QLGA_H */
