/*
 * rt.h -- C ABI of the GB300 adaptive ray-tracing library.
 *
 * The library computes the radiation field of point sources on a uniform
 * Cartesian grid with photon-conserving adaptive ray tracing (Wise & Abel,
 * arXiv:1012.2865, Sec. 2.1-2.2 and Steps 1-7 of Sec. 3.1) and the
 * hydrogen-only ionisation update that couples consecutive traces
 * (Eq. "dndt"), with the paper's optional features: the covering factor
 * (Sec. 2.3, RT_TRACE_FC), a finite speed of light with packages kept
 * between traces (Sec. 2.1, Step 3j, rt_trace_params.light_cm), H I / He I
 * / He II photon types (Sec. 3.2) and the adaptive timestep (Sec. 3.4,
 * rt_timestep).  All work runs in CUDA kernels on one GPU; there is no CPU
 * fallback.
 *
 * Conventions for every call:
 *   - return value: RT_OK (0) or one of the RT_ERR_* codes below; on error
 *     rt_get_last_error() gives a message (thread-local, valid until the
 *     next call on the same thread).  No exception crosses the ABI.
 *   - handles are opaque; the caller owns them and releases them with the
 *     matching *_destroy call.  A handle may be used from one host thread
 *     at a time; grids and batches of one context may be used from
 *     different threads (a batch and its member grids count as one handle).
 *   - a cell index is i + nx*(j + ny*k) (x fastest); all cells are cubes of
 *     width dx = box_len_cm / nx.
 *   - work is enqueued on the grid's CUDA stream (cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  Calls that return results
 *     to the host synchronise that stream; the others are asynchronous.
 *   - units: cm, s, photons/s, eV on input; k_ph in s^-1 and Gamma in erg/s
 *     per absorbing atom on output.
 */
#ifndef GB300_RT_H
#define GB300_RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RT_OK 0
#define RT_ERR_INVALID_ARG 1    /* argument out of range; nothing was changed */
#define RT_ERR_OOM 2            /* device memory could not be allocated */
#define RT_ERR_CUDA 3           /* a CUDA call failed (message has the CUDA error) */
#define RT_ERR_QUEUE_OVERFLOW 4 /* the package queue was too small (async traces only) */
#define RT_ERR_LEVEL_OVERFLOW 5 /* a package would exceed RT_MAX_LEVEL */
#define RT_ERR_TIMEOUT 6        /* a bounded device wait ran out; results are invalid */
#define RT_ERR_STATE 7          /* call not valid in the object's current state */

/* arithmetic of a grid */
#define RT_FP64 0        /* traversal, optical depth and deposits in FP64 */
#define RT_FP32_MIXED 1  /* traversal, tau and deposits in FP32 (geometry and
                            tau as FP32 pairs); FP64 photon budget; split,
                            crossing and termination decisions equal to the
                            FP64 ones (re-taken in FP64 near ties); the
                            ionisation update in FP32 with a double-float
                            Newton correction (~1e-13 of the FP64 one) */
/* where a caller buffer lives */
#define RT_MEM_HOST 0
#define RT_MEM_DEVICE 1
/* element type of a caller output buffer */
#define RT_DTYPE_F64 0
#define RT_DTYPE_F32 1

#define RT_MAX_LEVEL 14 /* pixel numbers 12*4^14 still fit 32 bits */

typedef struct rt_ctx rt_ctx;
typedef struct rt_grid rt_grid;
typedef struct rt_batch rt_batch;

/* Grid description (Sec. 2.2: the absorber density n_HI = n_H x_HI per cell). */
typedef struct {
  int nx, ny, nz;        /* cells per axis, each >= 1, nx*ny*nz < 2^31 */
  double box_len_cm;     /* x extent of the box (> 0) */
  int precision;         /* RT_FP64 or RT_FP32_MIXED */
  int mem_kind;          /* RT_MEM_HOST or RT_MEM_DEVICE for the arrays below */
  const double* n_H;     /* [ncell] hydrogen density, cm^-3, >= 0 */
  const double* x_HI;    /* [ncell] neutral fraction in [0, 1] */
  const double* x_HII;   /* [ncell] ionised fraction, or NULL for 1 - x_HI */
} rt_grid_desc;

/* Method parameters of one trace (Sec. 2.1). */
typedef struct {
  int level0;            /* initial HEALPix level of emitted packages (>= 0) */
  double phi_c;          /* minimum rays per cell face, Eq. "split" (> 0) */
  double f_term;         /* a package ends when P < f_term * P_0, (0, 1) */
  int max_level;         /* no split beyond this level (level0..RT_MAX_LEVEL) */
  int64_t queue_capacity;/* package records in the device queue; 0 = automatic */
  double timeout_s;      /* bound on any device-side wait; <= 0 = 2 s */
  int blocks_per_sm;     /* resident 256-thread blocks of the trace kernel per SM;
                            0 = as many as fit (lower it to share the GPU) */
  int segs_per_iter;     /* segments a lane traces between queue visits; 0 = tuned
                            (from the mean package length of the grid's last
                            trace read back: half of it, a power of two in [8, 64]) */
  int flags;             /* RT_TRACE_CHECKSUMS: also fill rt_budget.hashes;
                            RT_TRACE_FC: covering-factor correction */
  int passes;            /* launches over equal ranges of the sources (>= 0);
                            0 = 1, or as many as the automatic sizing needs */
  double light_cm;       /* finite speed of light (Sec. 2.1, Step 3j): c dt_P,
                            the distance light travels in this trace (cm,
                            >= 0); 0 = infinite speed of light.  See below. */
} rt_trace_params;
#define RT_TRACE_CHECKSUMS 1
/* Geometric correction (Sec. 2.3, Eqs. "midpoint", "fc"): each segment's
 * k_ph and Gamma contribution is scaled by f_c = (1/2 + D_edge / L_pix)^2,
 * capped at 1, with L_pix = r theta_pix the width of the package's pixel
 * (taken as a square, theta_pix = sqrt(4 pi / N_pix), r the radius where the
 * segment starts; f_c = 1 at r = 0) and D_edge the distance from the
 * segment's midpoint to the nearest face of the cell along the axes.  dP,
 * the photon budget and every decision are unchanged; k_ph is no longer
 * photon conserving (as the paper notes). */
#define RT_TRACE_FC 2
/* Self-test of the bounded waits: the trace also waits for one package that
 * never exists, so it cannot end by itself; its idle warps must give up
 * after timeout_s without progress and the trace return RT_ERR_TIMEOUT,
 * leaving the grid usable.  No other effect on the result's validity: the
 * trace's results are invalid (as after any RT_ERR_TIMEOUT). */
#define RT_TRACE_SELFTEST_STALL 4
/* Finite speed of light (light_cm > 0).  A package halts where light
 * emitted with it has travelled: a package emitted a traces ago halts at
 * radius rlim[a], rlim[0] = light_cm / dx and rlim[a] = the previous trace's
 * rlim[a - 1] + light_cm / dx (cell units, FP64).  The test follows the split
 * test and uses the crossing radius of the current cell; the cut segment is
 * deposited as usual and the termination test comes first.  The grid keeps
 * halted packages in device memory (photons/s, radius, optical depth, cell,
 * age); the next trace with light_cm > 0 continues them from their cells
 * through the medium of that trace, alongside the new packages of its
 * sources, and they do not count as created packages (counts, hashes).  The
 * store of halted packages grows by itself in a synchronous trace (out !=
 * NULL); an enqueued trace that fills it reports RT_ERR_QUEUE_OVERFLOW.  A
 * light_cm so short that more than 2^20 ages would be in flight is
 * RT_ERR_INVALID_ARG.  A trace with light_cm = 0, rt_clear_sources, and
 * adding the grid to a batch drop the packages in flight.  Batches and
 * rt_trace_noalloc trace with an infinite speed of light only (light_cm must
 * be 0). */

/* Result of a trace, per grid. */
typedef struct {
  double emitted;                      /* photons/s leaving the sources */
  double absorbed;                     /* photons/s absorbed in the grid */
  double escaped;                      /* photons/s leaving the box */
  uint64_t counts[RT_MAX_LEVEL + 1];   /* packages created per HEALPix level */
  uint64_t hashes[RT_MAX_LEVEL + 1];   /* order-free checksum of the created
                                          (source, level, pixel) set, see below;
                                          0 unless RT_TRACE_CHECKSUMS is set */
  uint64_t segments;                   /* cell segments with length > 0 */
  uint64_t fallbacks;                  /* FP32 crossing/split decisions re-taken in FP64 */
  uint64_t fallbacks_tau;              /* FP32 termination decisions re-taken in FP64 */
  uint64_t queue_pushed;               /* records written to the queue, all passes
                                          (children taken by a free lane of the
                                          splitting warp are not queued) */
  int status;                          /* RT_OK or the device-side error */
  float kernel_ms;                     /* duration of the trace launches themselves
                                          (CUDA events on the grid's stream) */
  uint64_t queue_peak;                 /* records of the largest pass */
  int passes;                          /* launches the sources were split into */
  double resumed;                      /* photons/s of the packages continued from
                                          the previous trace (light_cm > 0) */
  double halted;                       /* photons/s of the packages halted at c dt_P;
                                          emitted + resumed = absorbed + escaped + halted */
  uint64_t n_resumed, n_halted;        /* their numbers */
} rt_budget;

/* A package in flight between traces (finite speed of light), as returned by
 * rt_get_in_flight. */
typedef struct {
  double r_cm;          /* distance from its source */
  double P;             /* photons/s it carries */
  double tau;           /* optical depth accumulated since emission */
  int32_t src;          /* index of its source in the grid (order of addition) */
  int32_t level;        /* HEALPix level */
  uint32_t pix;         /* nested pixel number */
  uint32_t age;         /* traces since its emission */
  int32_t cell[3];      /* cell it halted in */
  int32_t pad;
} rt_flight;
/* hashes[l] is the sum modulo 2^64 over created packages of
 * mix(((uint64)src << 40) ^ ((uint64)l << 34) ^ pixel), where mix is the
 * 64-bit finaliser x ^= x>>31; x *= 0x7fb5d329728ea185; x ^= x>>27;
 * x *= 0x81dadef4bc2dd44d; x ^= x>>33.  src counts from 0 in the order the
 * grid's sources were added. */

/* Context: one CUDA device.  device >= 0.  It owns the pixel-direction
 * table of the FP32-mixed path (built on first use); its grids and batches
 * are destroyed before it. */
int rt_ctx_create(int device, rt_ctx** out);
int rt_ctx_destroy(rt_ctx* ctx);

/* Create a grid (Sec. 2.2 state: n_H, x_HI, x_HII) in library-owned device
 * memory.  The caller's arrays are copied; they may be freed on return.
 * n_H must be finite and >= 0 and x_HI in [0, 1] in every cell (checked on
 * the device; RT_ERR_INVALID_ARG names the first failing cell).
 * stream: cudaStream_t for all later work on this grid. */
int rt_create_grid(rt_ctx* ctx, const rt_grid_desc* desc, void* stream, rt_grid** out);
/* Wait for the grid's work, take it out of its batch (if any) and free its
 * device memory.  NULL is accepted. */
int rt_grid_destroy(rt_grid* grid);
/* Cells per axis of a grid (every per-cell array has nx*ny*nz elements). */
int rt_get_dims(rt_grid* grid, int* nx, int* ny, int* nz);

/* Append n point sources (Sec. 2.1, Step 1).  Host arrays, copied:
 *   pos_cm[3n] position in [0, box]^3, ndot[n] photons/s (>= 0),
 *   e_ph_eV[n] photon energy (>= 13.6), sigma_cm2[n] absorption cross section
 *   (>= 0).  Sources keep the order of addition (their index in hashes). */
int rt_add_sources(rt_grid* grid, int n, const double* pos_cm, const double* ndot,
                   const double* e_ph_eV, const double* sigma_cm2);
/* Remove every source; packages in flight (finite speed of light) are
 * dropped with them. */
int rt_clear_sources(rt_grid* grid);
/* Index of the grid's first source in the created-set checksum (default 0):
 * a grid that holds sources [first, first + n) of a larger set (one shard of
 * a source-partitioned trace) then contributes the same checksum terms as
 * the whole set traced in one grid.  first + number of sources <= 2^23. */
int rt_set_source_offset(rt_grid* grid, int first);
/* Set the emission rate of every source (n = number of sources, ndot[n]
 * photons/s >= 0), e.g. a time-varying luminosity such as Eq. "test12".
 * The next trace emits with the new rates; packages already in flight keep
 * the photons they were emitted with. */
int rt_set_source_rates(rt_grid* grid, int n, const double* ndot);
/* Copy the packages in flight after the last trace (finite speed of light)
 * into out[cap] (host memory); *n receives their number (all of them, also
 * when above cap).  Synchronous. */
int rt_get_in_flight(rt_grid* grid, rt_flight* out, uint64_t cap, uint64_t* n);

/* One radiative-transfer pass, Steps 1-5: zero k_ph and Gamma, emit
 * 12*4^level0 packages per source, trace every package through the grid
 * (DDA, Eq. "trace"; split, Eq. "split"; absorption, Eqs. "dtau", "flux";
 * deposits, Eqs. "kph", "gamma"; termination) and reduce the photon budget.
 * out == NULL: enqueue only (no host synchronisation; may be captured in a
 * CUDA graph when queue_capacity > 0); read the result with rt_get_budget.
 * out != NULL: wait; with queue_capacity 0, a trace that overflowed the
 * queue is redone with a larger queue, up to 2^31 records or half the free
 * device memory, and beyond that as several launches ("passes") over equal
 * ranges of the sources, which add into the same k_ph, Gamma and budget.  The
 * passes the sizing added (not params->passes) are kept as the start for the
 * grid's next trace.  A single source
 * whose packages do not fit returns RT_ERR_QUEUE_OVERFLOW.  A split hands
 * children 1-3 to free lanes of the same warp where it can and queues the
 * rest, so the records a trace queues vary a little from run to run; after a
 * successful one-pass trace with queue_capacity 0 the queue is grown to hold
 * every child of that trace's splits but child 0 (3/4 of the packages created
 * above level0), so that repeating it cannot overflow. */
int rt_trace(rt_grid* grid, const rt_trace_params* params, rt_budget* out);
/* Result of the last trace (synchronises the grid's stream). */
int rt_get_budget(rt_grid* grid, rt_budget* out);

/* Step 6: advance x_HI, x_HII of every cell by dt_s with nsub backward-Euler
 * substeps of Eq. "dndt" (hydrogen only, n_e = n_p = n_H x_HII, no
 * collisional ionisation), k_ph of the last trace held fixed, then refresh
 * the absorber density used by the next trace.  dt_s >= 0, nsub >= 1,
 * alpha_B >= 0 (cm^3/s).  Asynchronous. */
int rt_chem_update(rt_grid* grid, double dt_s, int nsub, double alpha_B);

/* Replace the gas state of every cell (Sec. 2.2): n_H (may be NULL to keep
 * it), x_HI, and x_HII (NULL for 1 - x_HI), in memory mem_kind, same checks
 * as rt_create_grid; refreshes the absorber density.  The new state is
 * staged and checked on the device: the call returns once the check is done
 * (the caller's arrays may then be reused) and leaves the state unchanged
 * when it fails. */
int rt_set_state(rt_grid* grid, const double* n_H, const double* x_HI, const double* x_HII,
                 int mem_kind);

/* Copy k_ph (s^-1), Gamma (erg/s) and x_HI of every cell into caller buffers
 * (any may be NULL) of element type dtype in memory mem_kind.  Synchronous. */
int rt_get_rates(rt_grid* grid, void* kph, void* gamma, void* x_HI, int dtype, int mem_kind);

/* The same two operations without waiting, for callers that overlap the
 * host<->device copies of one step with the kernels of the next (the
 * Sec. 2.2 state in, the Eqs. "kph", "gamma" rates out).  Not for grids in a
 * batch (RT_ERR_STATE).  The first call of either on a grid allocates its
 * staging area and streams (which synchronises the device).
 *
 * rt_set_state_async: as rt_set_state, but returns once the work is
 * enqueued.  Host arrays (best pinned) are copied on a stream of the
 * library's, concurrently with the grid's kernels -- x_HI and x_HII straight
 * into a second pair of state arrays that the grid swaps for its own once
 * the state is checked (the grid holds two copies of its state from the first
 * such call), n_H when given into a staging area -- and must stay unchanged
 * until that copy is done (rt_synchronize, or any call that waits for the
 * grid); device arrays are read in the grid's stream order.  The state is checked on the device as rt_set_state checks it; a
 * state that fails leaves the grid unchanged and is reported as
 * RT_ERR_INVALID_ARG, naming the first failing cell, by the next
 * rt_synchronize, rt_get_budget or waiting rt_trace (every trace enqueued
 * until the host has read the rejection carries that status).
 *
 * rt_get_rates_async: as rt_get_rates, but returns once the work is
 * enqueued.  The fields are taken at this point of the grid's stream (a
 * device-to-device snapshot into a staging area) and copied to host buffers
 * (best pinned) on a stream of the library's, concurrently with the grid's
 * later kernels; they are complete after rt_wait_rates or rt_synchronize.
 * Device buffers are filled in the grid's stream order.  A later
 * rt_get_rates_async waits on the device for this one's copies to leave the
 * staging area. */
int rt_set_state_async(rt_grid* grid, const double* n_H, const double* x_HI, const double* x_HII,
                       int mem_kind);
int rt_get_rates_async(rt_grid* grid, void* kph, void* gamma, void* x_HI, int dtype, int mem_kind);
/* Wait until the host copies of the last rt_get_rates_async are complete
 * (and only for those: the grid's kernels may still run). */
int rt_wait_rates(rt_grid* grid);
/* Copy x_HII likewise. */
int rt_get_ionised(rt_grid* grid, void* x_HII, int dtype, int mem_kind);

/* Photon types (Sec. 3.2).  Packages are monochromatic and of one type,
 * absorbed by that type's species only (Eq. "dtau" with its n_abs) and
 * depositing into that type's k_ph and Gamma (Eqs. "kph", "gamma", with
 * E_ph - E_i):
 *   RT_PHOTON_HI   0  n_abs = n_H x_HI (the grid state), E_i = 13.6 eV
 *   RT_PHOTON_HEI  1  n_abs = n_HeI,  E_i = 24.6 eV
 *   RT_PHOTON_HEII 2  n_abs = n_HeII, E_i = 54.4 eV
 * Every source starts as RT_PHOTON_HI.  The helium densities are inputs
 * (the helium network that would evolve them is the caller's);
 * rt_chem_update stays hydrogen-only and uses the H I rates. */
#define RT_PHOTON_HI 0
#define RT_PHOTON_HEI 1
#define RT_PHOTON_HEII 2
/* Helium absorber densities n_HeI[ncell], n_HeII[ncell] (cm^-3, finite,
 * >= 0; x fastest) in memory mem_kind, copied.  The first call allocates
 * their rates (and FP32 pairs on the mixed path).  Checked on the device
 * before anything changes (RT_ERR_INVALID_ARG names the first bad cell).
 * Synchronous. */
int rt_set_absorbers(rt_grid* grid, const double* n_HeI, const double* n_HeII, int mem_kind);
/* Photon type of every source (n = number of sources); a source's photon
 * energy must reach its type's threshold.  Types 1 and 2 need
 * rt_set_absorbers before the next trace (else RT_ERR_INVALID_ARG). */
int rt_set_source_types(rt_grid* grid, int n, const int* type);
/* k_ph (s^-1) and Gamma (erg/s) of photon type `type` per absorber of that
 * type, as rt_get_rates (type 0 = rt_get_rates' k_ph and Gamma). */
int rt_get_rates_typed(rt_grid* grid, int type, void* kph, void* gamma, int dtype, int mem_kind);
/* Adaptive radiative-transfer timestep (Sec. 3.4, Eqs. "dtelec",
 * "dtchange") from the grid's current k_ph and state: per cell
 * eps_ion / |k_ph + n_e alpha_B| (n_e = n_H (1 - x_HI), C_H = 0) in cells
 * "within the ionisation front", whose optical depth sigma_front n_HI dx
 * exceeds tau_front (the paper uses 0.5), dt_max elsewhere and at most
 * dt_max; smoothed by a 3x3x3 Gaussian of one cell width (weights
 * exp(-|d|^2/2), renormalised over the neighbours inside the grid); *dt_out
 * = the minimum over the grid, capped at 2 dt_prev when dt_prev > 0.
 * Computed in FP32 (relative error ~1e-6).  dt_max may be +inf.
 * Synchronous. */
int rt_timestep(rt_grid* grid, double eps_ion, double alpha_B, double sigma_front, double tau_front, double dt_max,
                double dt_prev, double* dt_out);

/* Overwrite k_ph and Gamma (the quantities rt_get_rates returns) with the
 * caller's arrays of element type dtype in memory mem_kind, converted to the
 * grid's precision: for a trace partitioned by sources over several grids or
 * devices, the sum of the partial rates is installed before rt_chem_update.
 * Synchronous for host arrays, stream-ordered for device arrays. */
int rt_set_rates(rt_grid* grid, const void* kph, const void* gamma, int dtype, int mem_kind);

/* ---------------------------------------------------------------------------
 * Batches: many grids traced by one persistent launch that shares one
 * package queue (Steps 1-5 for every grid at once), and one launch of the
 * ionisation update (Step 6) for every grid.  Each grid keeps its own fields,
 * photon budget and counters; results equal those of the grid traced alone
 * (up to the order of floating-point sums).  All grids of a batch have the
 * same precision and context.  Batch launches start after the work already
 * queued on each member grid's own stream (rt_set_state, say); per-grid calls
 * on a member wait for the batch's stream first.  Changes to a member's
 * sources (rates, types, offset) or absorbers take effect at the batch's
 * next launch (its tables and captured step are rebuilt).  Queue sizing and
 * source passes follow rt_trace.
 * ------------------------------------------------------------------------- */
/* stream: cudaStream_t for the batch's work; NULL = the batch creates its own
 * (a blocking stream). */
int rt_batch_create(rt_ctx* ctx, void* stream, rt_batch** out);
/* Wait for the batch's work and free it; its grids stay alive. */
int rt_batch_destroy(rt_batch* batch);
/* Add a grid; *slot receives its slot number (reused after removal).  A
 * grid is in at most one batch (RT_ERR_STATE otherwise); rt_grid_destroy
 * takes a grid out of its batch, rt_batch_destroy leaves its grids alive. */
int rt_batch_add(rt_batch* batch, rt_grid* grid, int* slot);
/* Take the grid in `slot` out of the batch (after the batch's work); the
 * slot is then free.  RT_ERR_INVALID_ARG for an empty slot. */
int rt_batch_remove(rt_batch* batch, int slot);
/* Number of grids in the batch. */
int rt_batch_size(rt_batch* batch);
/* One trace of every grid (as rt_trace; sync != 0 waits and retries a queue
 * overflow with a larger queue or more passes). */
int rt_batch_trace(rt_batch* batch, const rt_trace_params* params, int sync);
/* Ionisation update of every grid (as rt_chem_update).  Asynchronous. */
int rt_batch_chem(rt_batch* batch, double dt_s, int nsub, double alpha_B);
/* nsteps coupled steps (trace, then update) of every grid.  One step is
 * captured once as a CUDA graph (after a synchronous sizing trace) and
 * replayed; it is captured again when the grids or arguments change.
 * Asynchronous after the capture.  The graph keeps the sizing trace's pass
 * count; with queue_capacity 0 its queue holds 4x the largest pass's records
 * plus 2^20 (within the limit rt_trace states); a replay that needs more
 * reports RT_ERR_QUEUE_OVERFLOW through rt_batch_get_budget (its results are
 * then invalid). */
int rt_batch_step(rt_batch* batch, const rt_trace_params* params, double dt_s, int nsub, double alpha_B,
                  int nsteps);
/* Result of the last trace for the grid in `slot` (synchronises). */
int rt_batch_get_budget(rt_batch* batch, int slot, rt_budget* out);
/* Pick segs_per_iter and blocks_per_sm for this batch by timing traces
 * (CUDA events); writes them into *params. */
int rt_batch_autotune(rt_batch* batch, rt_trace_params* params);

/* Self-check of the FP32-mixed path's direction bound: the largest
 * |n32_i - n64_i| over all pixel centres of `level` (HEALPix, Step 3a),
 * computed on the device, and the bound the mixed path's decision bands
 * assume (*bound may be NULL).  Synchronous. */
int rt_selfcheck_directions(rt_ctx* ctx, int level, double* max_abs_err, double* bound);

/* Measurement aid (no counterpart in the paper): the rate at which device
 * `device` completes atomic reductions (RED) of 1 into an array of `words`
 * elements (a power of two in [2^10, 2^30]) of element type dtype
 * (RT_DTYPE_F32 or RT_DTYPE_F64), each to an element picked by a hash of
 * (thread, iteration) -- the scattered pattern of lanes following diverging
 * rays.  This is the roof of the trace's k_ph / Gamma deposits (Eqs. "kph",
 * "gamma") while the rate arrays stay in L2.  *reds_per_s receives the best
 * of five event-timed full-occupancy launches (after one warm-up).  The call
 * allocates and frees its array and its own stream; it is synchronous.
 * Errors: rt_probe_last_error() gives the message. */
int rt_probe_red(int device, int dtype, uint64_t words, double* reds_per_s);
/* Message for the last failed rt_probe_red on this host thread. */
const char* rt_probe_last_error(void);

/* ---------------------------------------------------------------------------
 * Allocation-free trace.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- applications
 * whose device memory is owned by a host framework (an arena or a caching
 * allocator with a fixed budget) and callers that must not let cudaMalloc or
 * cudaFree synchronise the device or change its memory footprint.
 *
 * It runs the same FP32-mixed trace as rt_trace on a grid the caller holds in
 * device memory, and keeps all scratch (package queue, control words, budget
 * sums and per-block budget rows, source records, a table of pixel
 * directions) in one static device
 * array of about 10 MiB that every device loading the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Limits: at most RT_NOALLOC_MAX_SOURCES sources and
 * RT_NOALLOC_MAX_RECORDS queue records per call (a larger trace returns
 * RT_ERR_QUEUE_OVERFLOW); queue_capacity, if set, must not exceed the latter;
 * the trace runs as one pass (params->passes 0 or 1).
 *
 * Every call shares the static array, and each call clears what must start
 * at zero; calls whose work overlaps on the GPU (other streams or host
 * threads) race on it and must be serialised by the caller.  The first call
 * on a device sets that device up (finds the array's device address, fills
 * the direction table) and synchronises the device: make it before any
 * stream capture.  The call is synchronous: it waits for the trace on
 * `stream` (cudaStream_t as void*, NULL = legacy default stream) and fills
 * *out.  Errors: rt_noalloc_last_error() gives the message.
 * ------------------------------------------------------------------------- */
#define RT_NOALLOC_MAX_SOURCES 1024
#define RT_NOALLOC_MAX_RECORDS 262144

typedef struct {
  int nx, ny, nz;        /* cells per axis, as in rt_grid_desc */
  double box_len_cm;     /* x extent of the box */
  const float* n_HI;     /* device [ncell]: FP32 rounding of n_H * x_HI */
  const double* n_H;     /* device [ncell]: hydrogen density (FP64 decisions) */
  const double* x_HI;    /* device [ncell]: neutral fraction (FP64 decisions) */
  float* kph;            /* device [ncell] output: k_ph, s^-1 (overwritten) */
  float* gamma;          /* device [ncell] output: Gamma, erg/s (overwritten) */
} rt_noalloc_grid;

int rt_trace_noalloc(const rt_noalloc_grid* grid, int nsrc, const double* pos_cm, const double* ndot,
                     const double* e_ph_eV, const double* sigma_cm2, const rt_trace_params* params,
                     void* stream, rt_budget* out);
/* Message for the last failed rt_trace_noalloc on this host thread. */
const char* rt_noalloc_last_error(void);

/* Wait for all work enqueued on the grid's stream (and for the copies of
 * rt_set_state_async / rt_get_rates_async); RT_ERR_INVALID_ARG if a state
 * uploaded by rt_set_state_async since the last report was rejected. */
int rt_synchronize(rt_grid* grid);

/* Number of kernels this library launched on the calling process so far. */
uint64_t rt_kernel_launches(void);

/* Message for the last error on this host thread ("" if none). */
const char* rt_get_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GB300_RT_H */
