/*
 * fv.h -- C ABI of the GB300 finite-volume library.
 *
 * One explicit first-order finite-volume time step on a 2D Cartesian grid,
 * as defined in Essadki et al., "A task-driven implementation of a simple
 * numerical solver for hyperbolic conservation laws" (arXiv:1701.05431):
 *   - problem statement: Sec. 2.1, Eq. (conservation_law) and
 *     Eq. (initial_condition): dW/dt + div F(W) = S(W), W in R^nVar;
 *   - mesh: Sec. 2.2, Nx x Ny cells on [xmin,xmax] x [ymin,ymax];
 *   - scheme: Sec. 2.2.1, Eq. (VF_scheme) with the Lax-Friedrichs flux and
 *     the stability condition Eq. (CFL_cond);
 *   - source: Sec. 2.2.2, Eq. (SourceTerm), first-order splitting;
 *   - partition: Sec. 3.2 (NPartX x NPartY balanced subdomains) and the
 *     overlap strips of Sec. 4.1.2;
 *   - systems: scalar advection; the Euler system of Sec. 5, Eq. (Euler);
 *     the evaporating-spray moment system of Sec. 6.1, Eq. (Essadki).
 *
 * Every step of the method runs in CUDA kernels on one GPU (sm_103a).  All
 * functions return an fv_status; none throws, exits or aborts.  Functions
 * taking a context are not thread-safe for the same context.
 *
 * Memory layout of every state array crossing this ABI: nVar planes, each
 * of Ny rows of Nx values, x fastest (var v of cell (i,j) at
 * v*Nx*Ny + j*Nx + i).  Cell (i,j) is centred at
 * (xmin + (i+1/2) dx, ymin + (j+1/2) dy).
 */
#ifndef FV_H
#define FV_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fv_status {
  FV_OK = 0,
  FV_ERR_INVALID_ARG = 1, /* bad argument or configuration                  */
  FV_ERR_CUDA = 2,        /* a CUDA runtime call failed (see fv_last_error) */
  FV_ERR_OOM = 3,         /* device allocation failed                       */
  FV_ERR_CFL = 4,         /* fixed dt violates Eq. (CFL_cond)               */
  FV_ERR_NONPHYSICAL = 5, /* rho <= 0, p <= 0, non-realizable moments, NaN  */
  FV_ERR_TIMEOUT = 6,     /* a bounded device wait ran out                  */
  FV_ERR_STATE = 7        /* call out of order (e.g. run before set_state)  */
} fv_status;

/* Systems (nVar in parentheses). */
enum { FV_ADVECTION = 0 /* (1) */, FV_EULER = 1 /* (4) */, FV_SPRAY = 2 /* (6) */ };

/* Storage and arithmetic precision of the state.
 *   FV_F64: FP64 storage and FP64 arithmetic;
 *   FV_F32: FP32 storage and FP32 flux/update arithmetic;
 *   FV_BF16: bfloat16 storage (rounded to nearest even after every step)
 *     with FP32 arithmetic; advection and Euler only, single instances only.
 * In every precision dt, t and the conservation totals are FP64, and the
 * spray source's maximum-entropy solve is FP64.  fv_set_state and
 * fv_get_state exchange FP64 or FP32 arrays in every precision. */
enum { FV_F64 = 0, FV_F32 = 1, FV_BF16 = 2 };

/* Boundary conditions, per side (Sec. 4.2, copyOverlaps):
 *   periodic: the wrapped neighbour cell (E must pair with W, N with S);
 *   transmissive: a copy of the border cell itself (zero gradient);
 *   dirichlet: the prescribed conserved state bc_state[side]. */
enum { FV_BC_PERIODIC = 0, FV_BC_TRANSMISSIVE = 1, FV_BC_DIRICHLET = 2 };
enum { FV_SIDE_E = 0, FV_SIDE_N = 1, FV_SIDE_W = 2, FV_SIDE_S = 3 };

/* Variable sets accepted by fv_set_state.
 *   FV_CONSERVED: W itself;
 *   FV_PRIMITIVE: advection (u); Euler (rho, u, v, p) with
 *     rho E = p/(gamma-1) + rho (u^2+v^2)/2; spray (m0, m1/2, m1, m3/2, u, v)
 *     with momenta m1 u, m1 v. */
enum { FV_CONSERVED = 0, FV_PRIMITIVE = 1 };

/* Problem statement (Sec. 2.1-2.2, 3.2).
 *   nx, ny >= 1; 1 <= npart_x <= nx, 1 <= npart_y <= ny (balanced split,
 *     the first Nx mod NPartX parts one cell wider); on one GPU the
 *     partition is realised as a tile work-list and does not change results.
 *   params: advection (a_x, a_y); Euler (gamma); spray (K, theta, gas field
 *     0: at rest / 1: Taylor-Green (sin 2pi x cos 2pi y, -cos 2pi x sin 2pi y),
 *     Q quadrature nodes (0 -> 32), Newton tolerance (0 -> 1e-13));
 *     theta <= 0 disables the drag term.
 *   cfl > 0 and fixed_dt <= 0: adaptive dt_n = cfl min(dx,dy)/lmax(W^n);
 *   fixed_dt > 0: the paper's constant dt, checked against Eq. (CFL_cond)
 *     at the start of every step (FV_ERR_CFL on violation).
 *   stream: cudaStream_t on which all work is queued (NULL: legacy stream).
 *   tune: 0 = the kernel the autotuner's recorded table names for this
 *     (system, precision, grid-size class, mode), or the occupancy
 *     heuristic where the table has no entry (fv_kernel_choice says which);
 *     1 = time the candidates at the first run and keep the fastest;
 *     >= 2: force candidate (tune - 2). */
typedef struct fv_config {
  int nx, ny, npart_x, npart_y;
  double xmin, xmax, ymin, ymax;
  int system;
  int precision;
  int bc[4];
  double bc_state[4][8];
  double cfl;
  double fixed_dt;
  double params[8];
  void *stream;
  int tune;
} fv_config;

typedef struct fv_ctx fv_ctx;

/* Static text for a status code. */
const char *fv_status_string(fv_status s);

/* Detail of the last failure on this context ("" if none; ctx may be NULL
 * for failures of fv_init). Owned by the library. */
const char *fv_last_error(const fv_ctx *ctx);

/* Validate cfg and allocate every device buffer (two state buffers of
 * nVar x Ny x pitch values -- 8 x Ny x pitch for FP64 Euler, whose kernels
 * also keep the primitives u, v, p, c of every cell -- and a control
 * block).  *out receives the context,
 * owned by the caller until fv_destroy.  FV_ERR_INVALID_ARG for a bad
 * configuration (unpaired periodic sides, non-positive sizes, unknown
 * system or precision), FV_ERR_OOM when allocation fails. */
fv_status fv_init(const fv_config *cfg, fv_ctx **out);

/* Release every device buffer and the context.  NULL is accepted. */
void fv_destroy(fv_ctx *ctx);

/* Load the state at t = 0, step 0 (initial condition,
 * Eq. (initial_condition)).  src: nVar x Ny x Nx values (layout above) of
 * type src_dtype (FV_F64 or FV_F32), on the device when src_is_device != 0
 * (any device pointer readable on the context's stream) else in host memory
 * (pinned or pageable).  The caller keeps ownership; the library copies.
 * Recomputes lmax(W^0) on the device.  Returns FV_ERR_NONPHYSICAL when the
 * state has rho <= 0, p <= 0, non-finite values or non-realizable moments,
 * and FV_ERR_INVALID_ARG when adaptive dt meets lmax = 0.  Synchronises the
 * stream. */
fv_status fv_set_state(fv_ctx *ctx, const void *src, int src_is_device, int src_dtype,
                       int layout);

/* Advance by one step (Eq. (VF_scheme) then Eq. (SourceTerm)); *dt_used
 * (nullable) receives the dt taken.  Same errors as fv_run. */
fv_status fv_step(fv_ctx *ctx, double *dt_used);

/* Advance by up to nsteps steps (one CUDA graph of nsteps fused step
 * kernels queued on the stream), stopping at t_end when t_end > 0 (the last
 * dt is clipped to land on t_end).  *t_out (nullable) receives the time
 * reached.  Error flags raised on the device are read back once at the end
 * (this synchronises the stream): FV_ERR_CFL (fixed dt too large; state kept
 * at the last good step), FV_ERR_NONPHYSICAL (the offending state is the
 * current state), FV_ERR_STATE when no state was set. */
fv_status fv_run(fv_ctx *ctx, int nsteps, double t_end, double *t_out);

/* Copy the current conserved state out as nVar x Ny x Nx values of
 * dst_dtype (FV_F64 or FV_F32), to device (dst_is_device != 0) or host
 * memory owned by the caller.  Synchronises the stream. */
fv_status fv_get_state(fv_ctx *ctx, void *dst, int dst_is_device, int dst_dtype);

/* Time blocking: steps_per_pass = 2 advances two time steps per kernel
 * launch, reading and writing the state once per two steps (half the bytes
 * per cell-update).  Needs the paper's fixed dt (fixed_dt > 0, Sec. 2.2.1),
 * advection or Euler, not in place; any boundary conditions (on a
 * transmissive or Dirichlet side the ghosts of the intermediate state take
 * the boundary condition inside the pass).  Results, times, step counts and
 * errors are bit for bit those of
 * one step per launch: a pass that finds the intermediate state failing the
 * paper's check dt lmax <= min(dx, dy) (or inadmissible) leaves everything
 * as it was and the steps from there run one at a time.  fv_run uses passes
 * when t_end <= 0 and at least two steps remain.  steps_per_pass = 1 turns
 * it off.  With tune >= 2 the (tune - 2)-th two-step kernel candidate is
 * used (FV_ERR_INVALID_ARG past the last one); otherwise the recorded
 * kernel table's two-step entry for the grid (tune = 0), else the first
 * candidate that fills the GPU.  Errors: FV_ERR_INVALID_ARG when a condition
 * above fails. */
fv_status fv_set_time_blocking(fv_ctx *ctx, int steps_per_pass);

/* In-place mode (on != 0; advection and Euler, every precision): the
 * context keeps ONE state buffer instead of two and updates it in place.
 * Each warp task writes, besides its cells, its border rows and columns of
 * W^{n+1} into overlap strips (the paper's ovlpE/N/W/S buffers, Sec. 4.1.2,
 * here filled by the task that produces the values, not by a copy task);
 * the next step reads its halo from its neighbours' strips, double-buffered
 * by step parity, so no task reads a value another is overwriting.  Results
 * are bit for bit those of the default mode.  Switching frees (on) or
 * allocates again (off) the second state buffer and keeps the current state,
 * time and step.  Autotuning (tune = 1) is not done in place; with
 * tune >= 2 the (tune - 2)-th in-place kernel candidate is used
 * (FV_ERR_INVALID_ARG past the last one); otherwise the recorded kernel
 * table's in-place entry for the grid (tune = 0), else the first candidate
 * that fills the GPU.  Errors: FV_ERR_INVALID_ARG (spray system),
 * FV_ERR_OOM, FV_ERR_CUDA. */
fv_status fv_set_inplace(fv_ctx *ctx, int on);

/* Asynchronous snapshot of the current state W^n, the counterpart of the
 * asynchronous output gathering of Sec. 4.3 (the solution is copied out for
 * writing while the time steps go on).  Queues on the context's stream a
 * copy of W^n into a device staging buffer owned by the context (converted
 * to dst_dtype, FV_F64 or FV_F32, in fv_get_state's layout), then, on a side
 * stream of the context, the copy of that buffer into dst, caller-owned HOST
 * memory of nVar * nx * ny values.  Returns without waiting; steps queued
 * afterwards (fv_run, fv_step) run while the host copy is in flight when dst
 * is pinned (page-locked) memory; with pageable memory the call returns only
 * after the copy.  dst must stay valid, and must not be read, until
 * fv_snapshot_wait returns.  A later snapshot waits on the device for the
 * previous host copy before it refills the staging buffer.
 * Errors: FV_ERR_INVALID_ARG (NULL dst, bad dtype), FV_ERR_STATE (no state),
 * FV_ERR_OOM, FV_ERR_CUDA. */
fv_status fv_snapshot(fv_ctx *ctx, void *dst, int dst_dtype);

/* Blocks until the last fv_snapshot's copy into host memory is complete
 * (FV_OK at once if none is pending). */
fv_status fv_snapshot_wait(fv_ctx *ctx);

/* Asynchronous input, the counterpart of fv_snapshot: queues on a side
 * stream of the context the copy of a state (fv_set_state's src layout,
 * nVar x Ny x Nx values of src_dtype, FV_F64 or FV_F32, conserved or
 * primitive per layout) from caller-owned HOST memory into a device buffer
 * owned by the context, and returns without waiting; with pinned memory the
 * copy runs while the steps already queued go on (pageable memory: the call
 * returns after the copy).  src must stay valid and unchanged until the
 * state is loaded by fv_set_state_prefetched.  A prefetch replaces one not
 * yet loaded; it waits on the device until the previous load has read the
 * buffer.  Errors: FV_ERR_INVALID_ARG (NULL src, bad dtype or layout),
 * FV_ERR_OOM, FV_ERR_CUDA. */
fv_status fv_prefetch_state(fv_ctx *ctx, const void *src, int src_dtype, int layout);

/* fv_set_state from the last fv_prefetch_state: the context's stream waits
 * on the device for the copy, then the state is loaded at t = 0, step 0 and
 * checked exactly as by fv_set_state (same results bit for bit, same errors;
 * synchronises the stream).  FV_ERR_STATE when no prefetch is pending. */
fv_status fv_set_state_prefetched(fv_ctx *ctx);

/* Per-variable totals sum_ij W_v dx dy of the current state (nVar doubles
 * into host memory), FP64 Neumaier-compensated block sums combined in a
 * fixed order (deterministic).  Synchronises the stream. */
fv_status fv_totals(fv_ctx *ctx, double *totals);

/* Simulation time and completed step count of the current state. */
fv_status fv_time(fv_ctx *ctx, double *t, long long *step);

/* Set the time and step counter of the current state (resume from a
 * checkpoint written with fv_get_state + fv_time). */
fv_status fv_set_time(fv_ctx *ctx, double t, long long step);

/* lmax(W^n) of the current state: the largest |eigenvalue| over cells and
 * the two axis normals, the quantity bounded by Eq. (CFL_cond). */
fv_status fv_lambda_max(fv_ctx *ctx, double *lmax);

/* Kernel variant in use: *variant receives its index, *desc (nullable) its
 * description such as "euler f32 v4 ty32 w4 b3 async4", followed by
 * ", 35-row tasks" when the rows per warp task were balanced away from the
 * kernel's nominal TY over the GPU's resident warps (the string stays valid
 * until the next call on ctx). */
fv_status fv_kernel_info(fv_ctx *ctx, int *variant, const char **desc);

/* Description of the two-step kernel fv_run uses (fv_set_time_blocking),
 * NULL when one step per launch is in force or ctx is NULL. */
const char *fv_kernel_info_two_step(const fv_ctx *ctx);

/* Description of compiled kernel candidate `index` (0-based) for a system
 * and precision, e.g. "euler f32 v1 ty64 w4 b6": V cells per lane, TY rows
 * per warp task, NW warps per block, register budget for b blocks per SM.
 * FV_ERR_INVALID_ARG past the last candidate.  fv_config.tune = index + 2
 * forces that candidate; tune = 1 times them all on the first fv_run. */
fv_status fv_kernel_candidate(int system, int precision, int index, const char **desc);

/* How the step kernel that fv_kernel_info names (two_step = 0), or the
 * two-step kernel (two_step != 0, FV_ERR_STATE when two steps per pass are
 * off), was chosen.  With fv_config.tune = 0 the library looks the
 * (system, precision, grid-size class, mode) key up in the table of choices
 * the autotuner recorded on a GB300 (python -m paper_1701_05431_gb300.autotune
 * times every candidate on a seeded workload of each measured class and
 * compiles the fastest into the library); *how is then "table: <key>
 * (<workload>, <rate> G cell-updates/s when recorded)".  Keys the table
 * lacks take the occupancy heuristic ("heuristic ...": the first candidate,
 * in order of preference, whose warp tasks fill the GPU).  tune = 1 gives
 * "autotuned ..." and tune >= 2 "forced ...".  Grid-size classes by cell
 * count: 0 below 2^16, 1 below 2^20, 2 below 2^24, 3 from 2^24 on.  The
 * string lives until the next call on the context. */
fv_status fv_kernel_choice(const fv_ctx *ctx, int two_step, const char **how);

/* Q-point Gauss-Legendre nodes x[Q] and weights w[Q] on [0,1] used by the
 * spray source's maximum-entropy quadrature (Sec. 6.2), as computed by the
 * library on the host.  1 <= Q <= 128. */
fv_status fv_gauss_legendre(int Q, double *x, double *w);

/* Measured FMA throughput of the current GPU (the denominator of the
 * arithmetic roofline).  The FP64 Euler step and the spray source step
 * (Sec. 6.2) are bound by the FP64 pipe rather than by HBM, so their
 * roofline fraction is the FP64 work they retire per second over this rate.
 * precision FV_F64 (DFMA) or FV_F32 (FFMA).  Every thread of a full grid
 * (8 blocks of 256 threads per SM) runs four, then eight, independent
 * a = a*b + c chains with register operands and no memory traffic; for each,
 * after a calibration launch, three launches of about `seconds` each
 * (0.001 <= seconds <= 2) are timed with CUDA events on `stream`, and
 * *fma_per_s receives the best of the six: thread-level FMA instructions
 * retired per second (FLOP/s = 2 x that).  Synchronises the stream;
 * allocates no device memory. */
fv_status fv_fma_peak(int precision, double seconds, double *fma_per_s, void *stream);

/* No-allocation totals.  The paper has no counterpart: this entry point is
 * for callers that cannot let the library allocate device memory (loops that
 * forbid allocator calls and the synchronisation they cause, frameworks that
 * own all device memory and account for every byte).  Same
 * per-variable totals sum_ij W_v * cell_area as fv_totals, for a caller-owned
 * device state of nvar x ny x nx values of dtype (FV_F64 or FV_F32, layout
 * above), written as nvar doubles to the caller's device buffer `totals`,
 * queued on `stream` without synchronising.  It calls no cudaMalloc, cudaFree
 * or allocating library routine: its partial sums use a fixed 128 KiB array
 * in the library's device image (per GPU, kept until the process exits), so
 * nvar is limited to 8 (FV_ERR_INVALID_ARG otherwise, with the reason in
 * fv_last_error(NULL)).  The first call on a device looks up that array's
 * device address with the device current; make that first call before any
 * stream capture.  All calls on a device share the array: calls that overlap
 * on the GPU race and must be ordered by the caller.  The looked-up address
 * is kept for the life of the process; after a cudaDeviceReset it no longer
 * names the array, so calls after a reset are not supported. */
fv_status fv_totals_noalloc(const void *state, int dtype, int nvar, int nx, int ny, double cell_area,
                            double *totals, void *stream);

/* ------------------------------------------------------------------------
 * Batched instances.  Many independent problems of the same system and
 * precision (advection or Euler; sizes, boundary conditions, parameters and
 * CFL may differ) advance together: one persistent kernel per fv_batch_run,
 * captured in a CUDA graph, takes warp tasks (instance, strip, rows) of all
 * instances and steps in a fixed increasing order; every instance keeps its
 * own dt_n = cfl min(dx,dy)/lmax(W^n) (Eq. (CFL_cond)) and t.  Each
 * instance's step is the same fused step as fv_run, with identical
 * arithmetic: an instance run in a batch gives the same bits as run alone.
 * Waits between the steps of an instance are bounded (2 s by default); a
 * wait that runs out ends the launch with FV_ERR_TIMEOUT.
 * ------------------------------------------------------------------------ */
typedef struct fv_batch fv_batch;

/* Validate n >= 1 configurations (same system, precision, stream and tune;
 * spray is not batched) and allocate every instance's two state buffers in
 * one device arena (FP64 Euler: 8 planes per buffer, the conserved variables
 * and the carried primitives u, v, p, c).  tune >= 2 forces batched kernel
 * candidate tune - 2. */
fv_status fv_batch_init(const fv_config *cfgs, int n, fv_batch **out);

/* Load instance k's state at t = 0, step 0 (same conventions as
 * fv_set_state).  Synchronises the stream. */
fv_status fv_batch_set_state(fv_batch *b, int k, const void *src, int src_is_device, int src_dtype,
                             int layout);

/* Advance every instance by nsteps steps in one persistent launch.  Returns
 * the first error raised by any instance (FV_ERR_CFL, FV_ERR_NONPHYSICAL,
 * FV_ERR_INVALID_ARG for lmax = 0) or FV_ERR_TIMEOUT; an instance that
 * failed keeps its last good state and stops advancing.  Synchronises. */
fv_status fv_batch_run(fv_batch *b, int nsteps);

/* Copy instance k's conserved state out (same conventions as
 * fv_get_state).  Synchronises the stream. */
fv_status fv_batch_get_state(fv_batch *b, int k, void *dst, int dst_is_device, int dst_dtype);

/* Time and step count of instance k. */
fv_status fv_batch_time(fv_batch *b, int k, double *t, long long *step);

/* Kernel candidate in use (see fv_kernel_info). */
fv_status fv_batch_kernel_info(fv_batch *b, int *variant, const char **desc);

/* Limit of every wait between steps (seconds, 0 < s <= 60) and, for tests
 * of the timeout path, an instance whose steps are never released
 * (-1: none); that instance's next step then waits until the limit and the
 * run returns FV_ERR_TIMEOUT without touching the GPU's health. */
fv_status fv_batch_set_wait_limit(fv_batch *b, double seconds, int never_release_instance);

/* Dataflow mode (on != 0): the instances advance with the paper's fixed dt
 * (Sec. 2.2.1) and, instead of one step-wide barrier per instance, every
 * warp task of step s waits only for its own and its neighbour tasks' step
 * s - 1 (the dependencies of the paper's task graph, Sec. 3.2, on the
 * device).  Results, times, step counts and errors are those of the default
 * step-gated mode, bit for bit: a task that finds dt lmax > min(dx, dy) on
 * cells it produced flags its instance, which is then put back to its state
 * at the start of the run (the library keeps one extra copy of every
 * instance's state for this) and replayed step-gated.  Requires fixed_dt > 0
 * for every instance (FV_ERR_INVALID_ARG otherwise); FV_ERR_OOM if the copy
 * cannot be allocated. */
fv_status fv_batch_set_dataflow(fv_batch *b, int on);

/* How the batched kernel was chosen, as fv_kernel_choice describes it (the
 * table is keyed by the cells of all instances together, mode "batched"). */
fv_status fv_batch_kernel_choice(const fv_batch *b, const char **how);

/* Detail of the last failure on this batch ("" if none). */
const char *fv_batch_last_error(const fv_batch *b);

/* Release every buffer of the batch.  NULL is accepted. */
void fv_batch_destroy(fv_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* FV_H */
