/*
 * librsst — GB300 (sm_103a) explicit finite-volume step of the reduced speed
 * of sound technique (RSST) for the Euler equations.
 *
 * Method: Iijima, Hotta & Imada, "Semi-conservative reduced speed of sound
 * technique for low Mach number flows with large density variations"
 * (arXiv:1812.04135).  One call of rsst_step advances the conserved state
 * U = (rho, m, E) by SSP-RK2 steps of the scheme of Sec. 4.2 (MUSCL with the
 * monotonized-central limiter, local Lax-Friedrichs flux with
 * c_tot = |V| + a/xi, CFL number 0.4), with the time derivative reduced by
 * one of the semi-conservative forms (Sec. 3.2 PVS; App. A DVS, PMS, DMS,
 * PD) and the external force of App. B.
 *
 * Conventions for every entry point:
 *  - Return value: RSST_OK (0) or a negative RSST_E* code; nothing aborts,
 *    prints or exits.  rsst_last_error() gives a message for the calling
 *    thread's last failure.
 *  - State layout seen by the caller (device or host memory, float64):
 *    structure of arrays [nvar][nz][ny][nx], x fastest, nvar = 2 + ndim,
 *    components (rho, m_x[, m_y[, m_z]], E).  Unused dimensions have size 1.
 *  - Buffers documented as device memory must be cudaMalloc'd or managed
 *    memory, host buffers (on_host = 1) pageable or pinned host memory; the
 *    kind is checked (cudaPointerGetAttributes) and a wrong one returns
 *    RSST_EINVAL before anything runs.  Sizes cannot be checked: a buffer
 *    must hold the layout stated for the call.
 *  - The caller owns every buffer it passes.  The library owns its working
 *    state (padded, with two ghost layers per active axis), its CFL scalars,
 *    flags, graphs and checkpoints; rsst_destroy frees them.
 *  - All GPU work is issued on the stream given to rsst_init (a
 *    cudaStream_t, NULL for the legacy default stream).  Calls documented
 *    as asynchronous return once the work is queued.
 *  - A handle (or batch) is not thread-safe: calls on one handle must not
 *    overlap; different handles may be used from different threads.
 *  - A non-physical state (rho <= 0, P <= 0 or a non-finite value) found
 *    by a step sets a sticky device flag; the next synchronous call returns
 *    RSST_ENONPHYSICAL.  The output is still written.  No floors are applied.
 *  - Every device wait of the TMA-staged kernels is bounded (2 s).  A wait
 *    that runs out sets a second flag bit: the kernel waits (bounded) for
 *    the copies it issued and returns, and the next synchronous call returns
 *    RSST_ETIMEOUT (reported before RSST_ENONPHYSICAL).  The context stays
 *    usable; rsst_set_state clears both bits.
 */
#ifndef RSST_H
#define RSST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSST_OK            0
#define RSST_EINVAL       -1  /* bad argument or configuration */
#define RSST_ECUDA        -2  /* a CUDA runtime/driver call failed */
#define RSST_ENONPHYSICAL -3  /* rho <= 0, P <= 0 or NaN/Inf produced */
#define RSST_ETIMEOUT     -4  /* a bounded device wait gave up */
#define RSST_EUNSUPPORTED -5  /* valid request the library does not provide */
#define RSST_ENOMEM       -6  /* device allocation failed */

/* Forms of the reduced time derivative (Sec. 3.2 and App. A). */
typedef enum {
  RSST_EULER = 0, /* no reduction: conservative Euler */
  RSST_DVS = 1,   /* "original" RSST, density reduced, App. A.1 */
  RSST_PVS = 2,   /* "semi-conservative", pressure reduced, Sec. 3.2 */
  RSST_DMS = 3,   /* momentum conserving, density reduced, App. A.3 */
  RSST_PMS = 4,   /* momentum conserving, pressure reduced, App. A.2 */
  RSST_PD = 5     /* mass and momentum conserving, App. A.4 */
} rsst_variant;

typedef enum {
  RSST_FP64 = 0,      /* state stored and computed in float64 (the two square
                       * roots of c_tot, which only set the LLF dissipation
                       * and dt, to 2^-40 relative; the LLF speed as a
                       * float pair on the float32 pipe) */
  RSST_FP32_PERT = 1, /* float32 perturbation about a float64 background */
  RSST_FP64_DF = 2    /* double-float: state stored and computed as pairs of
                       * float32 (hi + lo, 48-bit significand) on the float32
                       * pipe; float64 results to ~1e-13 at a fraction of the
                       * cost on GPUs with a slow float64 pipe */
} rsst_precision;

typedef enum { RSST_BC_PERIODIC = 0, RSST_BC_REFLECT = 1 } rsst_bc;

/* Run configuration.  Arrays are ordered (x, y, z); entries beyond ndim are
 * ignored.  The background (bg_rho, bg_p; HOST pointers, copied by
 * rsst_init) is a hydrostatic profile along axis `vertical` with
 * n[vertical] + 4 values: index k holds cell k - 2 (two ghost cells at each
 * end).  It sets the reflecting-wall ghost cells along `vertical`
 * (ghost = U0(ghost) + mirror(U - U0)(image), U0 = (rho0, 0, P0/(gamma-1)))
 * and, in RSST_FP32_PERT mode, the float64 state the float32 perturbation is
 * stored about.  With vertical = -1 there is no background (in
 * RSST_FP32_PERT mode the float32 state is then the full state).  On a
 * periodic vertical axis the ghost entries are ignored (taken by wrap).
 * rsst_init reads every entry it uses and rejects (RSST_EINVAL) one that is
 * not finite with rho > 0 and P > 0; it cannot check the arrays' length. */
typedef struct rsst_config {
  int32_t ndim;        /* 1, 2 or 3 */
  int32_t n[3];        /* interior cells per axis, >= 2 on active axes */
  double dx[3];        /* cell widths */
  int32_t bc[3];       /* rsst_bc per axis, both ends */
  int32_t variant;     /* rsst_variant */
  int32_t precision;   /* rsst_precision */
  double xi;           /* reduction rate, >= 1 (constant, Sec. 4.3) */
  double gamma;        /* ratio of specific heats */
  double cfl;          /* Courant number (0.4 in Sec. 4.2) */
  double grav[3];      /* constant acceleration F of App. B */
  int32_t vertical;    /* background axis, or -1 */
  int32_t cfl_rule;    /* 0: dt = cfl / max_cells sum_d c_tot/dx_d (default);
                        * 1: dt = cfl min_d dx_d / max_cells c_tot (the paper
                        * names only the Courant number, Sec. 4.2; in 1D the
                        * two agree) */
  const double* bg_rho;
  const double* bg_p;
  double cmax;         /* > 0: state-dependent reduction xi = [1 + (a/cmax)^4]^(1/4)
                        * (Eq. cx, Sec. 4.3) in c_tot and in f = 1 - 1/xi^2, per
                        * face state and per cell; 0: the constant xi above */
  double covolume;     /* equation of state (Sec. 3.2 states the reduced equations
                        * and dP for any EOS): 0 is the ideal gas; b > 0 the
                        * covolume (Noble-Abel) gas P = (gamma-1) e / (1 - b rho),
                        * a^2 = gamma P / (rho (1 - b rho)), e the internal energy
                        * per volume.  RSST_FP64 runs only (RSST_EUNSUPPORTED
                        * otherwise, and for the adjoint); a state with b rho >= 1
                        * is non-physical. */
} rsst_config;

typedef struct rsst_handle rsst_handle;

/* Create a solver for one run (the inputs of the scheme of Sec. 4.2: state,
 * form, xi, gamma, force, grid and walls).  Allocates the working state on
 * the current CUDA device; *h is NULL on failure and everything allocated is
 * freed.  `stream` is a cudaStream_t (may be NULL).  Errors: RSST_EINVAL for
 * an invalid config, checked before any device call (ndim, n, dx, bc, form,
 * precision, xi >= 1, gamma > 1, cfl > 0, cfl_rule 0 or 1, cmax >= 0,
 * covolume >= 0, finite gravity, the background entries, with b rho0 < 1);
 * RSST_EUNSUPPORTED for covolume > 0 in a precision other than RSST_FP64
 * (also checked first); RSST_ENOMEM when an allocation fails; RSST_ECUDA
 * when a copy, kernel or tensor-map encoding fails.  Synchronous. */
int rsst_init(rsst_handle** h, const rsst_config* cfg, void* stream);

/* Free everything the handle owns.  Safe on NULL.  Resource management: no
 * counterpart in the paper. */
void rsst_destroy(rsst_handle* h);

/* Load the full float64 state (caller layout above) from device memory
 * (on_host = 0) or host memory (on_host = 1), fill the ghost cells, clear
 * the non-physical flag and compute the CFL maximum of the new state.  U is
 * the conserved state (rho, m, E) of Sec. 3.2 that the update of Sec. 4.2
 * advances, as point values at cell centres.
 * Asynchronous for device input; host input is copied with cudaMemcpyAsync
 * (pinned memory keeps it asynchronous). */
int rsst_set_state(rsst_handle* h, const double* U, int on_host);

/* Write the full float64 state (background added back in RSST_FP32_PERT
 * mode) to device (on_host = 0) or host (on_host = 1) memory.  Synchronous
 * for host output; returns RSST_ENONPHYSICAL if the flag is set (the paper
 * applies no positivity floors; Sec. 4.2 has no such check, so this flag is
 * the library's). */
int rsst_get_state(rsst_handle* h, double* U, int on_host);

/* Advance nsteps SSP-RK2 steps (Sec. 4.2).  dt > 0: fixed step.  dt <= 0:
 * each step takes dt = cfl / max_cells sum_d c_tot/dx_d (cfl_rule 0; with
 * cfl_rule 1, cfl min_d dx_d / max_cells c_tot) from the state at
 * its start, entirely on the device.  Each step is two fused stage kernels
 * (reconstruction, LLF flux, divergence, RSST correction, force, RK update,
 * ghost cells; the second also reduces the CFL maximum).  Whole blocks of
 * rsst_set_graph_steps() steps replay a captured CUDA graph; the results
 * are the same as with plain launches.  Asynchronous. */
int rsst_step(rsst_handle* h, double dt, int nsteps);

/* Steps per replayed CUDA graph in rsst_step (default 16; 0 = plain
 * launches only).  k must be even and >= 0, else RSST_EINVAL.  A graph is
 * captured per CFL-slot parity on first use and again when a fixed dt
 * changes.  This is a launch-overhead control for small grids: the paper
 * has no counterpart. */
int rsst_set_graph_steps(rsst_handle* h, int32_t k);

/* The step the next adaptive rsst_step will take (cfl / CFL maximum of the
 * current state: the Courant condition of Sec. 4.2).  Synchronous. */
int rsst_dt(rsst_handle* h, double* dt_out);

/* Simulated time: the sum of the dt of the steps taken since the last
 * rsst_set_state (accumulated on the device).  Bookkeeping: no counterpart
 * in the paper.  Synchronous. */
int rsst_time(rsst_handle* h, double* t);

/* Wait for queued work; RSST_ENONPHYSICAL if a step flagged the state.
 * Stream control: no counterpart in the paper. */
int rsst_sync(rsst_handle* h);

/* Failure-detection test hook (no counterpart in the paper).  With
 * limit_ns > 0, from the next step on every tile of the TMA-staged stage
 * kernels also waits up to limit_ns on a shared-memory barrier that nothing
 * completes: in the 2D RSST_FP32_PERT kernel once its own copy has landed
 * (so no copy is in flight), in the 3D one after its first planes have
 * landed (the next plane's copy may still be in flight), and in the 2D/3D
 * RSST_FP64 kernel while its tile copy is in flight; a kernel waits for
 * copies it issued before leaving.  The wait runs out, the kernel sets the
 * run's timeout flag and returns without writing that tile, and the next
 * synchronous call returns RSST_ETIMEOUT; the state is then incomplete (load
 * one with rsst_set_state).  limit_ns = 0 restores normal steps.  Errors:
 * RSST_EINVAL unless 0 <= limit_ns <= 1e9; RSST_EUNSUPPORTED for runs that
 * do not use those kernels (they serve 2D RSST_FP32_PERT runs with vertical
 * axis y or none, 3D ones with vertical axis z or none, and 2D/3D RSST_FP64
 * runs).  Synchronous, launches nothing. */
int rsst_debug_stall_wait(rsst_handle* h, int64_t limit_ns);

/* Sum over cells of each conserved variable times the cell volume, in
 * float64, deterministic order (fixed-shape two-level tree): the totals whose
 * conservation by form Sec. 5 and App. A discuss.  In
 * RSST_FP32_PERT mode the background's sum (float64) is added to the sum
 * of the perturbation.  `sums` is host memory with nvar entries.
 * Synchronous. */
int rsst_conserved_sums(rsst_handle* h, double* sums);

/* ---- Discrete adjoint (float64 runs) ----------------------------------------
 * Reverse mode of the discrete SSP-RK2 step (transpose of the Jacobian of
 * U^n -> U^{n+1}; the paper gives the forward method only).  dt is held
 * fixed; non-smooth operations take the branch of the forward pass (MC
 * branch, LLF max with ties to the left state, zero subgradient of |V| at
 * V = 0).  Gradients are with respect to every component of the initial
 * conserved state and to xi. */

/* Run nsteps fixed-dt steps (Sec. 4.2) from the current state, storing a
 * checkpoint of the state every `every` steps (checkpointing has no
 * counterpart in the paper).  All device memory the adjoint needs is
 * allocated here (library-owned): ceil(nsteps/every) checkpoints, 2 x every
 * recompute states and their Euler tendencies, and a few state-sized work
 * arrays; RSST_ENOMEM if that fails.  The handle ends at U^{nsteps}.
 * RSST_EUNSUPPORTED for runs that are not float64 or not the ideal gas
 * (covolume > 0).  Asynchronous. */
int rsst_adjoint_record(rsst_handle* h, double dt, int nsteps, int every);

/* Number of recorded segments, ceil(nsteps / every) (no counterpart in the
 * paper).  RSST_EINVAL without a recorded run. */
int rsst_adjoint_segments(rsst_handle* h, int32_t* nseg);

/* Reverse segment `seg` (call from the last segment down to 0): recompute its
 * steps from the checkpoint, then apply the step adjoints in reverse (the
 * transpose of the Jacobian of the Sec. 4.2 step, a1-a9; no counterpart in
 * the paper).  lam:
 * device pointer, caller layout, float64; on entry dJ/dU at the segment's end,
 * on return dJ/dU at its start.  *dJ_dxi (host) is incremented by the
 * segment's contribution.  The handle's current state is preserved.
 * Allocates nothing.  Synchronous. */
int rsst_adjoint_step(rsst_handle* h, int32_t seg, double* lam, double* dJ_dxi);

/* J = sum_cells |m|^2/(2 rho) * cell volume of the current state (host
 * double) and, if grad is not NULL, dJ/dU into grad (device, caller layout:
 * (-|V|^2/2, V, 0) * cell volume).  The functional of the adjoint
 * conventions (no counterpart in the paper).  Float64 runs.  Synchronous. */
int rsst_kinetic_energy(rsst_handle* h, double* J, double* grad);

/* Density gradient at fixed velocity and pressure from a conserved-state
 * gradient (an option of this library's adjoint conventions; the paper has
 * no adjoint): with m = rho V and E = P/(gamma-1) + rho |V|^2/2,
 *   out = dJ/drho|_{V,P} = lam_rho + V . lam_m + |V|^2/2 lam_E
 * per cell, V from U.  U: the state the gradient refers to (the initial
 * state for rsst_adjoint_step's result), lam: dJ/dU, both device pointers,
 * float64, caller layout [ndim+2][nz][ny][nx] (no ghosts); out: device,
 * ncells float64; n: host array of ndim interior sizes.  Asynchronous on
 * `stream` (cudaStream_t, may be NULL).  RSST_EINVAL for NULL or host
 * pointers, ndim outside 1..3, n[d] < 1 or more than 2^31 cells. */
int rsst_adjoint_rho_fixed_vp(const double* U, const double* lam, double* out, int32_t ndim, const int32_t* n,
                              void* stream);

/* ---- Batched runs (one persistent kernel per RK stage for all runs) ------
 * Many independent 2D RSST_FP32_PERT runs (vertical axis y or none) of
 * uneven size, xi and background, advanced together (the method of Sec. 4.2
 * per run; batching is this library's, the paper runs one problem at a
 * time).  Each run keeps its own state, background tables and CFL dt, all on
 * the device.  The stream must be a created stream (the two stage launches
 * of a step are captured into a CUDA graph on it). */
typedef struct rsst_batch rsst_batch;

/* Create nruns runs from cfgs[0..nruns-1] (each as for rsst_init: the
 * inputs of the scheme of Sec. 4.2 per run).  Returns
 * RSST_EUNSUPPORTED for a run that is not 2D float32-perturbation with a y or
 * no vertical axis.  Synchronous. */
int rsst_batch_init(rsst_batch** b, int32_t nruns, const rsst_config* cfgs, void* stream);

/* Free every run and the batch's graphs and descriptors.  Safe on NULL.
 * Resource management: no counterpart in the paper. */
void rsst_batch_destroy(rsst_batch* b);

/* Per-run state transfer, as rsst_set_state / rsst_get_state (the state of
 * Sec. 3.2 per run).  RSST_EINVAL for a run index outside 0..nruns-1. */
int rsst_batch_set_state(rsst_batch* b, int32_t run, const double* U, int on_host);

/* See rsst_batch_set_state. */
int rsst_batch_get_state(rsst_batch* b, int32_t run, double* U, int on_host);

/* Advance every run nsteps adaptive SSP-RK2 steps of Sec. 4.2 (each with its own CFL dt):
 * per step one graph with two persistent launches over the ragged tile list
 * of all runs.  Asynchronous. */
int rsst_batch_step(rsst_batch* b, int nsteps);

/* The same steps (Sec. 4.2) with one pair of single-run launches per run per
 * step (the reference the persistent kernel is measured against). */
int rsst_batch_step_looped(rsst_batch* b, int nsteps);

/* Each run's next dt (nruns host doubles; the Courant condition of Sec. 4.2
 * per run).  Synchronous. */
int rsst_batch_dt(rsst_batch* b, double* dts);

/* Wait for every run's queued work and check every run's flag:
 * RSST_ETIMEOUT if a bounded device wait gave up in any run (the message
 * names the first such run and the count; a persistent block that gives up
 * flags every run whose tiles it leaves unwritten), else RSST_ENONPHYSICAL
 * if a run's state was flagged.  Stream control: no counterpart in the
 * paper. */
int rsst_batch_sync(rsst_batch* b);

/* rsst_debug_stall_wait for run `run` of a batch, in the persistent kernel
 * (no counterpart in the paper).  Waits for the batch's stream, then
 * rebuilds the run descriptors with the setting (graphs are recaptured on
 * the next step).  RSST_EINVAL for a bad run index or limit. */
int rsst_batch_debug_stall_wait(rsst_batch* b, int32_t run, int64_t limit_ns);

/* Time `steps` batch steps for each of six tile shapes (64x32, 32x32, 64x16,
 * 128x16, 64x24, 128x8 cells; index 0..5) on the current states (saved and
 * restored around the trials, also after a failed trial), keep the fastest;
 * *choice_out gets its index and *ms_out the milliseconds per step (either
 * may be NULL).  With RSST_TUNE_CACHE set to a file name the choice is read
 * from / appended to that file, keyed by the run list.  A performance
 * control: no counterpart in the paper.  Synchronous. */
int rsst_batch_autotune(rsst_batch* b, int steps, int32_t* choice_out, double* ms_out);

/* The tile shape in use, bx x by cells (host outputs).  No counterpart in the
 * paper.  RSST_EINVAL for NULL arguments. */
int rsst_batch_tile_shape(const rsst_batch* b, int32_t* bx, int32_t* by);

/* Number of kernels the batch launched so far (0 for NULL).  Bookkeeping:
 * no counterpart in the paper. */
int64_t rsst_batch_kernel_launches(const rsst_batch* b);

/* Conservation sums of a caller-held state, for callers that cannot allocate
 * device memory when they need them (inside another framework that owns the
 * device-memory budget; in loops that cannot take cudaMalloc's device
 * synchronisation).
 * The paper has no counterpart: it is a deployment convenience.
 *   U     device pointer, float64, caller layout [nvar][nz][ny][nx], read only
 *   ndim  1..3 (nvar = ndim + 2 <= 5); n, dx: host arrays of ndim entries
 *   sums  device pointer to nvar doubles, written with sum(U) * cell volume
 *   stream cudaStream_t (may be NULL); the call is asynchronous.
 * Allocates nothing: its only scratch is a file-scope device array of
 * 5 x 1024 doubles (40 KiB) that every GPU loading the library keeps until
 * exit.  The first call on a device looks that array's address up
 * (cudaGetSymbolAddress, with the device current) and keeps it for later
 * calls.  Calls share the array: two calls
 * that overlap on the GPU (different streams, not ordered) race and give wrong
 * sums.  Each call overwrites every scratch entry it reads, so no clearing is
 * needed.  Rejects ndim outside 1..3 and grids above 2^31 cells with
 * RSST_EINVAL.  Same reduction order as rsst_conserved_sums. */
int rsst_conserved_sums_noalloc(const double* U, int32_t ndim, const int32_t* n, const double* dx, double* sums,
                                void* stream);

/* Number of kernels the library launched through this handle so far (0 for
 * NULL).  Bookkeeping: no counterpart in the paper. */
int64_t rsst_kernel_launches(const rsst_handle* h);

/* Self-test of the float64 helpers the kernels use in place of compiler
 * sequences (no counterpart in the paper): over n seeded inputs, the largest
 * difference in ulps between the reciprocal (hardware seed and one
 * third-order step) and CUDA's correctly rounded 1.0/x (x in [2^-20, 2^20]);
 * the number of inputs on which the integer-pipe MC limiter differs from
 * the direct float64 form (plus 2^20 if a c_tot square root misses one of
 * its special cases: 0 and subnormal -> 0, negative and NaN -> NaN, or the
 * float-to-double bit conversion a case); and the largest relative
 * difference between either c_tot square root (the float64 one of the
 * adjoint and the C_max law, the float-pair one of the LLF speed and the CFL
 * rate) and CUDA's
 * sqrt (x in [2^-200, 2^200]).  All outputs are host pointers.
 * Synchronous, current device. */
int rsst_math_selftest(int32_t n, double* rcp_max_ulp, int32_t* mc_mismatches, double* sqrt_max_rel);

/* Float64 FMA throughput of the current device in TFLOP/s, measured by a
 * probe kernel (independent FMA chains on every SM, timed with CUDA events
 * after a warm-up launch; `iters` x 32 FMAs per thread), and the launch time
 * in ms (ms may be NULL).  The denominator of the float64 step's arithmetic
 * roofline: a performance measurement with no counterpart in the paper.
 * Synchronous, current device. */
int rsst_fp64_fma_peak(int32_t iters, double* tflops, double* ms);

/* sizeof(rsst_config) as compiled into the library (binding check; no
 * counterpart in the paper). */
size_t rsst_config_size(void);

/* Message describing the calling thread's most recent failure (thread-local
 * storage owned by the library; no counterpart in the paper). */
const char* rsst_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RSST_H */
