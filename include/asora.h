/*
 * asora.h -- C ABI of the GB300 short-characteristics ray tracer.
 *
 * Photo-ionisation rates from point sources on periodic 3-D hydrogen grids
 * (arXiv 2311.01492, "pyC2Ray"/ASORA): for every source, the H I column
 * density to each cell inside its ray-tracing radius is built by
 * short-characteristics interpolation from upstream cells plus the in-cell
 * path (Sec. 3.1, Eqs. raga/interp), converted to a photon-conserving rate
 * through tabulated transmission functions (Sec. 2.2, Eqs. gamma, tables,
 * sugg) and summed over sources.  A time-averaged chemistry update (Sec. 2.1,
 * Eq. time_avrg_sol) closes the ray-tracing <-> chemistry iteration (Fig. 1).
 *
 * Conventions (all entry points):
 *   - Every function returns rt_status; on failure rt_last_error() gives a
 *     thread-local message.  Nothing is partially applied on RT_ERR_INVALID.
 *   - Field pointers named d_* are DEVICE pointers of the current CUDA device,
 *     owned by the caller.  Inputs registered with rt_set_* are borrowed until
 *     the next rt_set_* of the same input or rt_grid_destroy; outputs are
 *     borrowed for the duration of the call (work is asynchronous on the
 *     grid's stream: the caller keeps buffers alive until that stream is
 *     synchronised).  Host pointers (h_*) are read during the call only.
 *   - Fields are FP64, C order: cell (i,j,k) of a box of size n is at
 *     (i*n + j)*n + k.  Ensembles concatenate boxes in box order.
 *   - Units are CGS: cm, s, cm^-3, cm^2.
 *   - The library owns all of its scratch memory (device) and frees it in
 *     rt_grid_destroy.  All work runs on the stream given at creation (or set
 *     with rt_set_stream); no call synchronises the device unless stated.
 */
#ifndef ASORA_H
#define ASORA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RT_OK = 0,
  RT_ERR_INVALID = 1, /* bad argument or bad input data                       */
  RT_ERR_OOM = 2,     /* device allocation failed                             */
  RT_ERR_CUDA = 3,    /* a CUDA runtime call failed                           */
  RT_ERR_TIMEOUT = 4, /* a bounded device-side wait ran out; no kernel of this version
                         waits on the device, so it is not returned              */
  RT_ERR_STATE = 5,   /* call order violated (e.g. trace before set_tables)   */
  RT_ERR_BOUNDS = 6   /* a device-side capacity or bounds check failed: the trace that
                         latched it is incomplete (reported by rt_check, rt_get_stats and
                         the calls that synchronise)                              */
} rt_status;

typedef struct rt_grid* rt_grid_t;
typedef void* rt_stream_t; /* a cudaStream_t; NULL = legacy default stream */

/* Physics parameters.  rt_params_default() fills the paper's values. */
typedef struct {
  double sigma0_cm2; /* H I cross section at threshold, 6.3e-18 cm^2 (Sec. 4.1.3)         */
  double tau_lim;    /* cells with dtau*ds <= tau_lim use the thin limit (Eq. gammalocal)  */
} rt_params;

/* Trace schedules for rt_raytrace. */
enum {
  RT_SCHED_AUTO = 0,    /* batched (autotuned or default configuration), or plain if the autotuner found it faster */
  RT_SCHED_PLAIN = 1,   /* ASORA-style: one CTA per source, octahedral shells S_q in order   */
  RT_SCHED_BATCHED = 2, /* persistent work queue over (source, face, quadrant) items, LPT   */
  RT_SCHED_BATCHED_EXIT = 3 /* as BATCHED, but an item stops once a whole layer is opaque
                               (tau_out >= 2^E1 (1+2^-40) everywhere): the rates are the same
                               bit for bit, the skipped column densities are not computed    */
};

/* Interpolation weights of Eq. interp (rt_set_interpolation). */
enum {
  RT_INTERP_GEOMETRIC = 0,   /* the paper's geometric (bilinear) weights, Sec. 3.1 (default) */
  RT_INTERP_OPTICAL_DEPTH = 1 /* geometric weights modulated by 1/max(tau_n, tau_weight_min) and
                                 normalised, after the C2Ray paper's App. A, to which Sec. 3.1
                                 refers for the weighting: favours the less opaque interpolants */
};

/* Rate table kinds for rt_set_tables. */
enum {
  RT_TABLE_CHORDS = 0, /* chords through knot values of g and h (Eq. tables)                */
  RT_TABLE_GREY_EXACT = 1 /* grey opacity evaluated exactly: g = h = exp(-tau) (Sec. 4.1.1)  */
};

void rt_params_default(rt_params* p);

/* Thread-local message describing the last failure of this thread. */
const char* rt_last_error(void);

/* One periodic box of n^3 cells of size cell_cm.  s: stream for all work. */
rt_status rt_grid_create(rt_grid_t* g, int n, double cell_cm, const rt_params* p, rt_stream_t s);

/* An ensemble of nbox independent periodic boxes (h_n[b]^3 cells of size
 * h_cell_cm[b]) traced in one launch.  Fields are the boxes concatenated. */
rt_status rt_ensemble_create(rt_grid_t* g, int nbox, const int* h_n, const double* h_cell_cm,
                             const rt_params* p, rt_stream_t s);

rt_status rt_set_stream(rt_grid_t g, rt_stream_t s);

/* Number of knots of a table with parameters (E0, E1, bits): (E0+E1)*2^bits + 2.
 * Knot 0 is tau = 0, knot 1+t is 2^(t>>bits - E0) * (1 + (t & (2^bits-1))/2^bits),
 * the last knot is 2^E1.  tau >= 2^E1 transmits nothing. */
int rt_table_nknots(int E0, int E1, int bits);

/* Knot values of the frequency-integrated transmission g(tau) = gamma(N_HI)/Ndot
 * (Eq. tables normalised by Eq. ngammalnu) and h(tau) = -dg/dtau for a blackbody of
 * temperature T_bb (K) with sigma_nu = sigma0 (nu/nu_th)^-beta, h nu_th = 13.6 eV
 * (Sec. 2.2, 4.1.3).  Host arrays of rt_table_nknots() doubles.  Host code. */
rt_status rt_table_blackbody(double T_bb, double beta, int E0, int E1, int bits, double* h_g,
                             double* h_h);

/* Rate tables (host arrays of rt_table_nknots(E0,E1,bits) doubles, copied).
 * kind RT_TABLE_CHORDS: g, h are knot values; a lookup of tau uses segment
 * 1 + (e+E0)*2^bits + m from tau's binary exponent e and top mantissa bits m
 * (segment 0 below 2^-E0) and returns fma(c1, tau, c0) with
 * c1 = (v_hi - v_lo)/(tau_hi - tau_lo), c0 = fma(-c1, tau_lo, v_lo).
 * kind RT_TABLE_GREY_EXACT: g and h may be NULL; exp(-tau) is used. */
rt_status rt_set_tables(rt_grid_t g, int kind, int E0, int E1, int bits, const double* h_g,
                        const double* h_h);

/* Hydrogen density n_H (cm^-3) and neutral fraction x_HI of every cell.
 * Validated (finite, n_H >= +0, 0 <= x_HI <= 1, no negative zero): this call
 * synchronises the grid's stream and returns RT_ERR_INVALID on bad data. */
rt_status rt_set_density(rt_grid_t g, const double* d_nH);
rt_status rt_set_xHI(rt_grid_t g, const double* d_xHI);

/* Expanding background (Sec. 4.1.2, Test 2: comoving grid, density diluted by
 * the expansion).  From this call on, the cell sizes given at creation and the
 * densities given to rt_set_density are comoving values at scale factor 1: the
 * ray trace and the chemistry use the proper cell size cell * a and the proper
 * density n_H * a^-3, with a^-3 evaluated as 1 / (a * a * a) and the products
 * rounded once each.  Rates are proper (s^-1), column densities proper (cm^-2).
 * a = 1 (the default) reproduces the static results bit for bit.  a must be
 * finite and in [1e-6, 1e6] (RT_ERR_INVALID otherwise).  Applies to every box of
 * an ensemble; synchronises the grid's stream. */
rt_status rt_set_scale_factor(rt_grid_t g, double a);

/* Sources: d_pos int32[nsrc][3] cell indices (i,j,k) in [0,n), d_box int32[nsrc]
 * box ids (NULL: all in box 0), d_ndot photon rates (s^-1, >= 0), d_radius
 * ray-tracing radius in cells (> 0; cells with |Delta|^2 > floor(R^2) are not
 * traced, Sec. 3.3).  Sources in the same cell with the same radius are merged by
 * summing their rates (Sec. 3: identical spectra).  The library copies what it
 * needs; the pointers are not kept.  Synchronises the grid's stream.  On failure
 * (RT_ERR_INVALID, RT_ERR_OOM, ...) the grid holds no sources until the next
 * successful call (a trace then writes zero rates). */
rt_status rt_set_sources(rt_grid_t g, int nsrc, const int32_t* d_pos, const int32_t* d_box,
                         const double* d_ndot, const double* d_radius);

/* Photo-ionisation rate Gamma (s^-1) of every cell, summed over all sources,
 * written to d_gamma (all cells overwritten).  schedule: RT_SCHED_*. */
rt_status rt_raytrace(rt_grid_t g, double* d_gamma, int schedule);

/* Column density (cm^-2) from source `src` (index in the rt_set_sources arrays)
 * through the far side of every traced cell; 0 outside its traced region.
 * schedule: RT_SCHED_PLAIN or RT_SCHED_BATCHED/AUTO (same values bit for bit). */
rt_status rt_raytrace_source_coldens(rt_grid_t g, int src, double* d_coldens, int schedule);

/* Chemistry step (Sec. 2.1, Eq. time_avrg_sol) for every cell, isothermal
 * hydrogen.  d_x0: x_HII at the start of the step; d_xavg_in: time-averaged x_HII
 * used by the ray trace that produced d_gamma.  Iterates n_e = n_H <x_HII> until
 * |change| <= tol*<x> (tol = 1e-10) or 50 iterations.  Writes <x_HII> to
 * d_xavg_out and x_HII(t+dt) to d_xnew_out; adds to *d_unconverged (device int64)
 * the number of cells whose neutral fraction 1-<x> moved by more than
 * conv_tol (relative) from 1 - d_xavg_in. */
rt_status rt_chemistry_step(rt_grid_t g, const double* d_gamma, const double* d_x0,
                            const double* d_xavg_in, double dt_s, double alpha_H, double C_H,
                            double conv_tol, double* d_xavg_out, double* d_xnew_out,
                            int64_t* d_unconverged);

/* One time step of the ray-tracing <-> chemistry iteration (Fig. 1): starting
 * from <x> = x0 (d_x, x_HII, updated in place to x(t+dt)), repeat
 * {x_HI = 1-<x>; Gamma = trace; <x> = chemistry} until fewer than
 * conv_frac * ncells cells are unconverged or max_iter iterations.  With
 * use_graph != 0 the max_iter iterations are one captured CUDA graph whose
 * later iterations are no-ops once converged; the graph is kept and replayed by
 * later calls with the same d_x, d_gamma, dt_s, alpha_H, C_H, max_iter,
 * conv_tol, conv_frac and stream when no rt_set_*, rt_autotune or
 * rt_set_schedule call came in between (otherwise it is captured again).  d_gamma receives the last
 * rates; *h_iters (host, may be NULL) the iterations run (synchronises).
 * Requires rt_set_density; the grid's registered x_HI is replaced by an
 * internal buffer. */
rt_status rt_iterate(rt_grid_t g, double* d_x, double dt_s, double alpha_H, double C_H,
                     int max_iter, double conv_tol, double conv_frac, int use_graph,
                     double* d_gamma, int* h_iters);

/* Adjoint of rt_raytrace for L = sum_p w_p Gamma_p with w = d_dL_dgamma (n^3):
 * writes dL/dlog n_HI of every cell to d_dL_dlog_nHI (n^3, overwritten) and
 * dL/dlog Ndot of every input source to d_dL_dlog_ndot (nsrc, overwritten;
 * members of a merged source share its derivative in proportion to their
 * rates).  n_HI = n_H x_HI enters through dtau and the 1/n_HI of Eq. sugg; the
 * table lookups are differentiated as the chords they are (exact grey: exp).
 * Column densities are recomputed per (source, face) item, never stored per
 * source.  The thin/thick switch is treated as locally constant. */
rt_status rt_raytrace_backward(rt_grid_t g, const double* d_dL_dgamma, double* d_dL_dlog_nHI,
                               double* d_dL_dlog_ndot);

/* Interpolation weights of every later trace (batched and plain schedules and
 * rt_raytrace_source_coldens): RT_INTERP_GEOMETRIC (default) or
 * RT_INTERP_OPTICAL_DEPTH, where each interpolant's geometric weight w_n becomes
 * w_n / max(tau_n, tau_weight_min) (tau_n its optical depth at threshold,
 * sigma0 N_HI) and tau_in = sum(w'_n tau_n) / sum(w'_n), both sums in the order
 * n = 1..4 of the geometric chain.  tau_weight_min finite and > 0 (0.6 is the
 * binding's default).  The adjoint supports the geometric weights only (rt_raytrace_backward
 * returns RT_ERR_INVALID otherwise).  RT_ERR_INVALID for other modes. */
rt_status rt_set_interpolation(rt_grid_t g, int mode, double tau_weight_min);

/* Adjoint recompute mode: with stop_at_opaque != 0 (default) each item's
 * recompute stops at its first layer whose cells all have tau_out >= 2^E1 (1+2^-40);
 * every later tau_in is then >= 2^E1, every later rate exactly 0, and no gradient
 * flows from there, so the result is the same.  0 recomputes every layer. */
rt_status rt_set_adjoint_mode(rt_grid_t g, int stop_at_opaque);

/* Timing/launch statistics of the last rt_raytrace on this grid (device event
 * time of the trace kernels, launches, source-voxels traced). */
typedef struct {
  double trace_ms;          /* event time of the trace kernel launches              */
  double prep_ms;           /* event time of per-call preparation (dtau, zeroing)   */
  int64_t source_voxels;    /* sum over (merged) sources of traced cells            */
  int64_t items;            /* work items of the last launch                        */
  int64_t rate_cells;       /* (source, cell) pairs whose rate was evaluated (tau_in below
                               the table's upper bound; elsewhere the rate is exactly 0) */
  int64_t kernel_launches;  /* rt_kernel_launch_count() at the time of the call         */
  int launches;             /* kernel launches of the last rt_raytrace              */
  int schedule;             /* schedule used                                        */
  int block;                /* threads per CTA of the trace kernel                  */
  int grid;                 /* CTAs of the trace kernel                             */
  int64_t row_table_bytes;  /* precomputed row tables of the ingested radii (0: none) */
} rt_stats;

/* Schedule of RT_SCHED_BATCHED: (face, quadrant) items of sources whose largest
 * layer half-width exceeds hsmall are traced by CTAs of block_big threads (128 or
 * 256), the others by single warps (hsmall 0..32; 0 = CTAs only); of those,
 * sources whose largest layer half-width is at most hface (0..20; 0 = off) have
 * each face traced whole by one warp (every cell of a face once, no cell shared
 * between quadrants).  rt_raytrace_backward uses block_big CTAs of 128 and
 * min(hsmall, 27) (its warps hold more shared memory).  Defaults 128, 19, 13;
 * results do not depend on the choice. */
rt_status rt_set_schedule(rt_grid_t g, int block_big, int hsmall, int hface);

/* Autotuner of RT_SCHED_BATCHED: times rt_raytrace on the registered fields and
 * sources for block_big in {128, 256} x hsmall in {0, 11, 15, 19, 22, 24, 27, 30}
 * (whole-face warps off), then hface in {9, 11, 13, 15, 17, 19} at the fastest pair, then
 * hsmall again at that hface; keeps the fastest and returns it in *h_block, *h_hsmall,
 * *h_hface (any may be NULL).
 * Finally times the plain (block-per-source) schedule once: RT_SCHED_AUTO takes
 * whichever of the two is faster.  With a cache file (may be NULL), a line
 * "<workload key> <block> <hsmall> <hface> <auto_plain>" whose key (box sizes,
 * source count and radius distribution) matches is used without timing, and a
 * new result is appended.  Synchronises; allocates one temporary rate field. */
rt_status rt_autotune(rt_grid_t g, const char* cache_path, int* h_block, int* h_hsmall,
                      int* h_hface);

/* Statistics of the last trace (synchronises the grid's stream).  Fills *out,
 * then returns RT_ERR_BOUNDS if a kernel latched a failed device-side check
 * since the last report (see rt_check). */
rt_status rt_get_stats(rt_grid_t g, rt_stats* out);

/* Device-side checks.  The trace kernels check their own capacities (layer
 * width against the shared-memory buffers, layer index against the geometry
 * table, source extent against the plain schedule's cube); a failed check
 * skips the rest of that work item and latches an error bit in the grid
 * instead of touching memory out of bounds.  Kernels run asynchronously, so
 * rt_raytrace and rt_raytrace_backward return before such a bit can be seen:
 * rt_check synchronises the grid's stream and returns RT_ERR_BOUNDS (and clears
 * the bits) if any is latched, RT_OK otherwise.  rt_get_stats,
 * rt_raytrace_source_coldens and rt_iterate with h_iters, which synchronise
 * anyway, report the same. */
rt_status rt_check(rt_grid_t g);

/* Failure injection for tests: latches error bits (1 = layer capacity, 2 =
 * geometry table, 4 = input data, 8 = plain-schedule cube) in the grid's
 * device-side error word as a failed check would; no kernel runs.
 * Synchronises.  RT_ERR_INVALID for other bit values. */
rt_status rt_inject_device_error(rt_grid_t g, int bits);

/* Process-wide cap on the device memory this library holds (all grids and
 * scratch, every device), in bytes; 0 removes the cap.  The environment
 * variable ASORA_DEVICE_MEMORY_LIMIT sets the initial cap.  An allocation that
 * would exceed it fails as an out-of-memory would (RT_ERR_OOM), before calling
 * cudaMalloc; the grid stays usable (see rt_set_sources for what a failed
 * source ingest leaves).  Negative values: RT_ERR_INVALID. */
rt_status rt_set_device_memory_limit(int64_t bytes);

/* Device memory this library holds right now (bytes, all grids). */
int64_t rt_device_memory_in_use(void);

void rt_grid_destroy(rt_grid_t g);

/* Column density (cm^-2) from one source through every traced cell, exactly as
 * rt_raytrace_source_coldens computes it (bit for bit), for callers that cannot
 * allocate device memory when they call: code running while someone else
 * captures a CUDA graph, frameworks that reserve all device memory at start-up
 * and forbid cudaMalloc afterwards, or loops where an allocation's implicit
 * synchronisation is not acceptable.  The paper has no counterpart; it is the
 * plain (octahedral-shell) trace of one source with its scratch cube in a fixed
 * file-scope device array instead of library-allocated memory.
 *   n, cell_cm, sigma0_cm2 : box size, cell size (cm), threshold cross section
 *   d_nH, d_xHI            : device fields (n^3, C order), read only, not validated
 *   i, j, k, radius        : source cell and radius in cells (> 0)
 *   d_coldens              : device output, n^3 doubles, fully overwritten
 *   s                      : stream (NULL = legacy default stream)
 * Allocates nothing: no cudaMalloc/cudaFree and no allocating library call.  The
 * traced half-extent min(floor(R), n/2) must not exceed 40 cells (the scratch
 * array holds one 81^3 cube, 4.25 MB, reserved on every GPU that loads the
 * library until the process exits); larger requests return RT_ERR_INVALID
 * before launching anything.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current: make it
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents (every cell a call reads it has written first); calls that
 * overlap on the GPU race on it, so serialise them. */
rt_status rt_coldens_single_noalloc(int n, double cell_cm, double sigma0_cm2, const double* d_nH,
                                    const double* d_xHI, int i, int j, int k, double radius,
                                    double* d_coldens, rt_stream_t s);

/* Number of CUDA kernels this library has launched from host code in this
 * process (kernels replayed by a CUDA graph are counted when captured). */
long long rt_kernel_launch_count(void);

/* Cells of the octahedral shell S_q = {|Di|+|Dj|+|Dk| = q} (Sec. 3.3, App. A) in
 * the order the RT_SCHED_PLAIN kernel assigns them to threads: the top part
 * Dk >= 0 (2q(q+1)+1 cells) then the bottom part.  Writes 3 ints per cell to
 * h_out (host, may be NULL) and returns |S_q| = 4q^2+2 (1 for q = 0), or -1 for
 * q < 0.  Host code, no GPU needed. */
int rt_shell_enumerate(int q, int32_t* h_out);

#ifdef __cplusplus
}
#endif

#endif /* ASORA_H */
