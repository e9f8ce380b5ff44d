/*
 * hybro_place.h -- C ABI of the GB300 (sm_103a) electrostatic global-placement
 * library: the inner loop that every perturb-and-reoptimise round of Hybro
 * re-runs (the global-placement step of Algorithm 1, run until it converges),
 * plus the perturbations (Shuffle, Shuffle (all), WireMask; Section 4.2) and
 * best-result selection of Algorithm 1, and a job server.
 *
 * Conventions
 *  - Every function returns PLACE_OK (0) or a negative PLACE_E* code; the
 *    message of the last failure on the calling host thread is returned by
 *    place_last_error() (borrowed, valid until the next failing call on that
 *    thread).
 *  - A handle owns a private device copy of the netlist and all device state.
 *    Handles are not thread-safe: use one handle per host thread.
 *  - All device work is issued on the stream given at creation (a
 *    cudaStream_t passed as void*; NULL = legacy default stream).  Functions
 *    that return results to host memory synchronise that stream.
 *  - "host or device" pointers are copied with cudaMemcpyDefault (unified
 *    addressing); the caller keeps ownership of every pointer it passes.
 *  - A handle holds K independent copies of the design ("copies", Algorithm 1
 *    restarts run as a batch); copy c is 0..K-1.  Copies share the netlist and
 *    the fixed cells; each has its own positions, optimiser state, density map
 *    and spectral buffers.
 *  - Layouts: cell arrays are [n_cells] with movable cells first; bin maps
 *    are x-major, element (ix, iy) at ix * ny + iy.
 */
#ifndef HYBRO_PLACE_H
#define HYBRO_PLACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PLACE_OK 0
#define PLACE_EINVAL (-1)    /* malformed argument or netlist */
#define PLACE_ENOMEM (-2)    /* device or host allocation failed */
#define PLACE_ECUDA (-3)     /* a CUDA call failed */
#define PLACE_ERANGE (-4)    /* design does not fit the fixed-point range */
#define PLACE_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define PLACE_EINTERNAL (-6) /* a device-side check failed */

/* Perturbation operators of Algorithm 1 (Section 4.2). */
#define PLACE_SHUFFLE_MACRO 0 /* Shuffle: p% of the movable macros */
#define PLACE_SHUFFLE_ALL 1   /* Shuffle (all): p% of all movable cells */
#define PLACE_WIREMASK 2      /* WireMask: every movable macro in turn to the
                                 grid position of least HPWL */

/* Spectral-solve arithmetic. */
#define PLACE_DCT_AUTO (-1) /* the default: PLACE_DCT_BF16X3 when nx and ny are
                               multiples of 128, else PLACE_DCT_FP32 */
#define PLACE_DCT_FP32 0   /* FP32 CUDA-core GEMMs (any grid, multiples of 16) */
#define PLACE_DCT_BF16X3 1 /* split-BF16 (3 products, FP32 accumulation) on the
                              tcgen05 tensor cores; grids must be multiples of 128 */

typedef struct place_t place_t;

/* Netlist N = (V, E) of Section 3 (Preliminaries).  Host pointers.
 * Cells [0, n_movable) move; the rest are fixed.  x0/y0 are lower-left
 * corners (initial positions for movable cells, final for fixed ones).
 * Net e owns pins net_ptr[e] .. net_ptr[e+1]-1; pin j sits on cell
 * pin_cell[j] at offset (pin_dx[j], pin_dy[j]) from the cell's lower-left.
 * net_w (nullable: all 1) weights a net in HPWL (Eq. 1) and WL (Eq. 2).
 * is_macro (nullable: none) marks the macros: Shuffle picks among the movable
 * ones and WireMask moves them. */
typedef struct place_netlist {
  int32_t n_cells, n_movable, n_nets, n_pins;
  const float *w, *h, *x0, *y0;
  const int32_t *net_ptr;
  const int32_t *pin_cell;
  const float *pin_dx, *pin_dy;
  const float *net_w;
  const uint8_t *is_macro;
} place_netlist;

/* Placement region [xl, xh) x [yl, yh).  xl, yl and the bin size must be
 * exact multiples of 2^-F for the fixed-point resolution F chosen at create
 * (any die with integer or dyadic-rational bounds qualifies).  F is the
 * largest value <= 24 with max(|xl|, |yl|, |xh|, |yh|, xh - xl, yh - yl) 2^F
 * < 2^30 and (total cell area) 2^2F < 2^62. */
typedef struct place_die { double xl, yl, xh, yh; } place_die;

/* nx x ny density bins and the target density t of the overflow test
 * (D(s) <= epsilon in Eq. 1).  nx and ny are multiples of 16 up to 8192; the
 * tensor-core spectral path needs multiples of 128. */
typedef struct place_bins { int32_t nx, ny; float target_density; } place_bins;

/* Optimiser constants.  The paper cites, but does not restate, the
 * Nesterov optimiser and the lambda/gamma schedules of DREAMPlace/ePlace; the
 * defaults from place_default_params() are this library's reading:
 *   gamma_k = gamma_base * w_bin * 10^((20/9) tau_{k-1} - 11/9)  (Eq. 3's gamma)
 *   lambda_0 = lambda_eta * |grad WL|_1 / |grad D|_1            (Eq. 2's lambda)
 *   lambda_{k+1} = lambda_k * clamp(mu_base^(1 - dHPWL/dref), mu_lo, mu_hi),
 *     dref = hpwl_ref * n_nets * w_bin
 *   alpha_0 = alpha0 * w_bin / rms(g_0); then |dv| / |dg|
 *   stop when overflow <= tau_stop (tau_stop < 0: never) or after max_iters.
 * Backtracking (max_backtracks > 0; ePlace's step-length prediction with
 * backtracking).  At k >= 1 the estimate |v_k - v_{k-1}| / |g_k - g_{k-1}|
 * also tests the step that led to v_k.  Below 0.95 times that step's length,
 * the step is redone from v_{k-1} with the estimate as its length, at most
 * max_backtracks times in a row.  lambda, gamma and k advance only on accepted
 * steps.  The overflow stop test applies at every evaluated point.  It costs
 * 8 bytes per movable cell and copy.
 * Density stretching (stretch = 1; ePlace's local smoothing).  Along each
 * axis, a movable cell narrower than sqrt(2) bins widens to
 * W' = rint(sqrt(2) BW) in fixed point, about its centre: the left edge
 * moves by floor((W' - W) / 2).  Its density is scaled by
 * R = floor(W H 2^31 / (W' H')) / 2^31.  Each (cell, bin) term of this second
 * map is floor(overlap R), exact in integers.  The stretched map drives the
 * field and the density gradient, which is scaled by R.  The overflow, the
 * stop test and gamma keep the exact unstretched map.  It costs 8 bytes per
 * bin and copy and 20 bytes per movable cell.
 * Filler cells (fillers = 1; ePlace's whitespace fillers).  Pinless movable
 * cells that take up the whitespace the target density leaves, so that the
 * density force holds the real cells together at the target density instead
 * of spreading them over the die.  Their size is the mean quantised width
 * and height of the movable non-macro cells, each rounded to a multiple of
 * 2^-F; their count floor(max(0, t (A_die - A_fixed) - A_mov) / (w_f h_f)),
 * with A_fixed the fixed area inside the die; their start uniform over the
 * die from a SplitMix64 stream.  They enter the density that drives the field
 * and every optimiser norm, never the HPWL, the WA model, the overflow or a
 * perturbation; a reset keeps them where they are.  place_get_fillers returns
 * them; place_info.n_fillers counts them. */
typedef struct place_params {
  int32_t n_copies;       /* K >= 1 */
  float gamma_base;       /* 4 */
  float lambda_eta;       /* 1e-3 */
  float alpha0;           /* 0.05 */
  float hpwl_ref;         /* 0.3 */
  float mu_base, mu_lo, mu_hi; /* 1.1, 0.95, 1.05 */
  float tau_stop;         /* 0.07 */
  int32_t max_iters;      /* 1000 */
  float constant_gamma;   /* > 0: fixed gamma (tests) */
  int32_t dct_mode;       /* PLACE_DCT_AUTO (default), _FP32 or _BF16X3 */
  int32_t max_backtracks; /* 0 (off) .. 64: redo a too-long step at most this
                             often in a row (see below) */
  int32_t stretch;        /* 0 (off) or 1: density stretching (see below) */
  int32_t autotune;       /* 1 (default): the knobs below left at their automatic
                             value are chosen by timing candidates on this design
                             at create (results cached per shape in the process);
                             0: fixed rules */
  int32_t scatter_mode;   /* -1 (default): the density scatter picks per copy and
                             pass, from the previous pass's effective number of
                             occupied bins, between merging a warp's shared bins,
                             a shared-memory table and direct atomics; 0, 1, 2
                             force one of them.  All give the same map. */
  int32_t gemm_bn;        /* 0 (default): automatic; 64 or 128: tile width of
                             every tensor-core GEMM stage of the spectral solve */
  int32_t wa_big_cap;     /* 0 (default): automatic; 32..6144: pins of a net of
                             more than 256 pins kept in shared memory */
  int32_t gemm_split;     /* 0 (default): automatic; 1: one CTA per GEMM tile;
                             2: two CTAs per 128-wide tile, one half of the
                             contraction each, on stages with at most half as
                             many tiles as the device has SMs.  Every choice
                             gives the same bits. */
  int32_t fillers;        /* 0 (default) or 1: filler cells (see below) */
  float macro_precond;    /* 1 (default): weight of a movable macro's charge in
                             its preconditioner, max(1, pins_i + k lambda area_i)
                             with k = macro_precond for macros, 1 otherwise;
                             above 1 a macro moves in shorter steps than the
                             standard cells around it */
  int32_t wa_streams;     /* 0 (default): automatic; 1, 2 or 3: the WA degree
                             classes run as a chain on one graph branch, or
                             split over two or three branches that run side by
                             side (integer gradient sums: the same bits) */
  int32_t dct_fold;       /* 1 (default): on the BF16x3 path with both grid sides
                             multiples of 256, every transform is split into its
                             even and odd frequencies (the first step of a fast
                             cosine transform), which halves the tensor-core
                             work of the solve; 0: the plain GEMMs.  Both solve
                             the same Poisson equation (to rounding). */
} place_params;

/* Read-only facts about a handle. */
typedef struct place_info {
  int32_t n_cells, n_movable, n_nets, n_pins, nx, ny, n_copies;
  int32_t frac_bits;      /* F: coordinates are quantised to multiples of 2^-F */
  int64_t bin_w_q, bin_h_q; /* bin size in units of 2^-F */
  double bin_w, bin_h;
  int64_t device_bytes;   /* device memory the handle holds */
  int32_t kernels_per_iter; /* this library's kernel launches in one iteration (the first
                              iteration after a reset adds one: k_precond0) */
  int32_t dct_mode;       /* the spectral path in use: PLACE_DCT_FP32 or _BF16X3 */
  int32_t n_fillers;      /* filler cells (0 unless params.fillers) */
  int32_t bounds_checked; /* 1: the library was built with index checks
                           * (-DPLACE_DEBUG_BOUNDS): a failed check makes the
                           * next synchronising call return PLACE_EINTERNAL */
  int32_t gemm_bn[4];     /* tile width of each tensor-core GEMM stage */
  int32_t gemm_split[4];  /* CTAs per tile of each stage (split-K when 2) */
  int32_t wa_big_cap;     /* pins of a big net kept in shared memory */
  int32_t autotuned;      /* 1: the choices here came from timing (or its cache) */
  double scatter_t1, scatter_t2; /* effective-bin thresholds of the scatter's ways */
  double autotune_ms;     /* host time the tuning took at create (0 on a cache hit) */
  int32_t wa_streams;     /* graph branches the WA classes run on (1..3) */
  int32_t dct_fold;       /* 1: the solve runs the even/odd split (params.dct_fold) */
} place_info;

/* Optimiser scalars of one copy after its last iteration. */
typedef struct place_state {
  int32_t iter;        /* iterations done since the last reset */
  int32_t converged;   /* 1: stopped by the overflow test */
  int32_t stopped;     /* 1: converged or reached max_iters */
  int32_t backtracks;  /* steps redone since the last reset */
  double lambda, gamma, alpha, a;
  double overflow;     /* tau at the current reference point */
  double hpwl_wa;      /* HPWL measured in the last iteration's WA pass */
  double bins_effective; /* (sum M)^2 / sum M^2 over the movable-area map of the
                          * last density pass: the effective number of occupied
                          * bins (0 before the first pass).  Below 256 the
                          * density scatter merges the lanes of a warp that hit
                          * the same bin; the map is the same either way. */
} place_state;

/* One accepted Nesterov iteration of one copy (place_get_history). */
typedef struct place_iter_record {
  int32_t iter;        /* k: iterations done before this one since the last reset */
  int32_t backtracks;  /* steps redone since the last reset, up to this one */
  double hpwl_wa;      /* HPWL at v_k from the iteration's WA pass (FP32 pins) */
  double overflow;     /* tau at v_k (exact, Eq. 1's density constraint) */
  double lambda;       /* the density weight of Eq. 2 for the next iteration */
  double gamma;        /* Eq. 3's gamma for the next iteration */
  double alpha;        /* the step length this iteration took */
} place_iter_record;

void place_default_params(place_params *p);

/* Create a handle: validates and copies the netlist (host pointers), chooses
 * the fixed-point resolution F, builds the device state for K copies (all
 * starting at x0/y0) and resets their optimisers.  Section 3 (problem
 * statement), the initial placement of Algorithm 1.  *out receives the
 * handle; on failure it is set to NULL and nothing is leaked.
 * PLACE_ERANGE: the die, a cell or the total area does not fit the 64-bit
 * density fixed point, or a movable cell carries so many pins that its
 * wirelength-gradient sum (accumulated as 32-bit fixed point with a scale
 * 2^Fg, Fg >= 10, from the bound 3 + 2 ln(degree) per pin and unit net
 * weight) would not fit. */
int place_create(const place_netlist *nl, const place_die *die, const place_bins *bins,
                 const place_params *params, void *stream, place_t **out);

/* Release every resource of the handle (NULL is ignored). */
int place_destroy(place_t *h);

int place_get_info(const place_t *h, place_info *out);

/* Run up to n_iters Nesterov iterations of Eq. 2 on every active copy (the
 * global-placement step of Algorithm 1).  With backtracking, n_iters counts
 * gradient evaluations, and a redone step is one of them.  A copy stops
 * updating once converged or at max_iters; the others continue.  converged
 * (nullable, host [K]) receives the stopped flags, which synchronises the
 * stream; with NULL the call is asynchronous. */
int place_step(place_t *h, int32_t n_iters, int32_t *converged);

/* place_step over n resident handles at once, as a job server would: the
 * iterations are launched round-robin, one per handle per round, each on its
 * handle's stream, so handles created on distinct streams run concurrently
 * (handles sharing a stream run one after another, with the same results).
 * hs: host [n] handles.  converged (nullable, host [sum of the handles' K])
 * receives the stopped flags, handle by handle, which synchronises every
 * handle's stream; with NULL the call is asynchronous.  EINVAL on a NULL
 * handle or n < 1; nothing is launched then. */
int place_step_multi(place_t *const *hs, int32_t n, int32_t n_iters, int32_t *converged);

/* Perturb (the perturbation step of Algorithm 1; Section 4.2) copy `copy`
 * (-1: every copy), then fully reset the optimiser of the perturbed copies.
 *
 * Shuffle / Shuffle (all): strength p in [0, 1].  Selection draws
 * SplitMix64 keys from `seed`; with copy -1, copy c uses seed + c.
 *
 * PLACE_WIREMASK ignores p and seed; it is deterministic.  The movable macros
 * (is_macro) move one at a time, by decreasing area (ties by index), each to
 * the bin corner that minimises the weighted HPWL (Eq. 1) of its nets.  The
 * other pins stay where they are; macros moved earlier count at their new
 * places.  A macro stays inside the die and off every fixed cell and every
 * macro moved before it; touching edges is allowed.  Ties go to the smallest
 * L1 distance from the macro's old corner, then the lowest bin row, then the
 * lowest column.  A macro with no free corner stays where it is.  The first
 * WireMask call allocates device scratch of about
 * 8 K (nx + ny + 8 max_nets_per_macro) + 20 K min(nx ny / 256, 304) bytes,
 * freed by place_destroy.  It runs four small kernels per macro, captured
 * into a CUDA graph on the first call for each copy selection and replayed
 * by later calls (the graph is freed by place_destroy).  A design
 * without movable macros only resets the optimiser.  EINVAL on an unknown
 * op or, for Shuffle, p outside [0, 1]; ENOMEM if the scratch cannot be
 * allocated. */
int place_perturb(place_t *h, int32_t op, float p, uint64_t seed, int32_t copy);

/* Exact FP64 HPWL (Eq. 1) and overflow of every copy at its current
 * positions: hpwl, overflow are host [K] (either may be NULL).  Synchronises. */
int place_eval_hpwl_overflow(place_t *h, double *hpwl, double *overflow);

/* Positions of copy `copy`: x, y are [n_cells] host or device buffers. */
int place_get_positions(place_t *h, int32_t copy, float *x, float *y);

/* Filler positions of copy `copy` (lower-left corners): x, y are host or
 * device float buffers of at least cap entries (either may be NULL);
 * min(cap, n_fillers) are written and *n (nullable) receives n_fillers.
 * Synchronises. */
int place_get_fillers(place_t *h, int32_t copy, float *x, float *y, int32_t cap, int32_t *n);

/* Set the filler positions of copy `copy` (-1: all copies) from [n_fillers]
 * host or device arrays, clamp them into the die and reset that copy's
 * optimiser (as place_set_positions does).  A no-op without fillers. */
int place_set_fillers(place_t *h, int32_t copy, const float *x, const float *y);

/* Borrowed device pointers to the positions of copy `copy`, valid until
 * place_destroy.  The library keeps each copy's positions interleaved,
 * (x_0, y_0, x_1, y_1, ...), so that every pin costs one 8-byte gather: cell
 * i is (*x)[2 i], (*y)[2 i], for i < n_cells.  With filler cells the library
 * orders its cells movable, fillers, fixed: fixed cell i (i >= n_movable) is
 * then at entry i + n_fillers.  Reads must be ordered after
 * the handle's work on its stream; the arrays belong to the library and may
 * not be written (place_set_positions does that). */
int place_device_views(place_t *h, int32_t copy, float **x, float **y);

/* Set the movable positions of copy `copy` (-1: all copies) from [n_cells]
 * host or device arrays (entries >= n_movable are ignored), clamp them into
 * the die and reset that copy's optimiser. */
int place_set_positions(place_t *h, int32_t copy, const float *x, const float *y);

int place_get_state(place_t *h, int32_t copy, place_state *out);

/* Per-iteration records of copy `copy` since its last reset (a placement's
 * convergence: HPWL, overflow, lambda, gamma, step length per iteration).  The
 * device keeps the last PLACE_HISTORY_CAP records per copy in a ring, written
 * by the iteration's last kernel; out (host, nullable) receives the last
 * min(cap, kept) of them, oldest first, and *n (nullable) their number.
 * Synchronises. */
#define PLACE_HISTORY_CAP 4096
int place_get_history(place_t *h, int32_t copy, place_iter_record *out, int32_t cap, int32_t *n);

/* Checkpoint of one copy's optimiser state, for pausing a placement and
 * resuming it on this handle or on a new handle of the same design, grid and
 * parameters: the positions u and v (fillers included), the previous
 * reference point, both gradient buffers and the raw gradients, the pending
 * WA sums, the backtracking arrays when on, the scalars (lambda, step length,
 * momentum, gamma, overflow, iteration count, stop flags) and the history
 * ring.  A placement resumed from it continues bit for bit as if it had not
 * been interrupted (the kernels are deterministic).
 * place_checkpoint_bytes: the size of one copy's checkpoint.
 * place_checkpoint_save: writes it to the host buffer buf of cap bytes
 *   (PLACE_EINVAL when smaller).
 * place_checkpoint_load: replaces copy `copy`'s state; PLACE_EINVAL when the
 *   buffer is short or its header (sizes, grid, fixed-point resolution, the
 *   lambda schedule's reference step, the knobs that add arrays) differs from
 *   this handle's.  Both synchronise. */
int place_checkpoint_bytes(const place_t *h, int64_t *bytes);
int place_checkpoint_save(place_t *h, int32_t copy, void *buf, int64_t cap);
int place_checkpoint_load(place_t *h, int32_t copy, const void *buf, int64_t bytes);

/* ---- stage-level evaluation at the current positions of one copy --------
 * These run the same kernels as place_step on the copy's reference point
 * v and leave the optimiser state untouched (the stage buffers they use are
 * overwritten). */

/* Eq. 3 summed over nets in x and y with the given gamma: *wl (host,
 * nullable) and grad_x/grad_y ([n_movable] host or device, nullable), the
 * gradient with respect to the movable lower-left corners. */
int place_eval_wirelength(place_t *h, int32_t copy, float gamma, double *wl,
                          float *grad_x, float *grad_y);

/* Movable-cell density map M (int64, units of 2^-2F, [nx*ny] x-major,
 * host or device, nullable) and the overflow tau (host, nullable). */
int place_eval_density(place_t *h, int32_t copy, int64_t *map, double *overflow);

/* The stretched map of copy `copy` from its last density pass (int64,
 * units of 2^-2F, [nx*ny] x-major, host or device).  Every density pass
 * (an iteration, place_eval_density, place_eval_field) writes it beside M.
 * Synchronises.  EINVAL when the handle was created without stretching. */
int place_get_stretched_map(place_t *h, int32_t copy, int64_t *map);

/* Fixed-cell map F (int64, [nx*ny], host or device). */
int place_get_fixed_map(place_t *h, int64_t *map);

/* Spectral Poisson solve of rho = (M + t F) / A_bin at the current positions
 * (M: the stretched map when density stretching is on): psi, ex, ey are
 * [nx*ny] host or device float buffers (nullable). */
int place_eval_field(place_t *h, int32_t copy, float *psi, float *ex, float *ey);

/* Density gradient -sum_b a_ib E_b for the movable cells using the field of
 * the current positions: grad_x/grad_y [n_movable] host or device.  With
 * density stretching, a_ib is the stretched rectangle's overlap times the
 * cell's density scale. */
int place_eval_density_grad(place_t *h, int32_t copy, float *grad_x, float *grad_y);

/* Hybro (Algorithm 1) on every copy: rounds 0..n_rounds place each copy until
 * convergence, record (HPWL, overflow), and perturb the current solution with
 * `op`, `p` and seed + round * K + copy before the next round.  The best
 * solution of each copy by (overflow <= tau_target, HPWL, overflow, round)
 * is kept on the device.  best_hpwl, best_overflow, best_round: host [K],
 * nullable.  Synchronises. */
int place_hybro(place_t *h, int32_t n_rounds, int32_t op, float p, uint64_t seed,
                float tau_target, double *best_hpwl, double *best_overflow,
                int32_t *best_round);

/* Best positions kept by place_hybro for copy `copy` ([n_cells], host or device). */
int place_get_best_positions(place_t *h, int32_t copy, float *x, float *y);

/* Per-round record of the last place_hybro call for copy `copy`: the exact
 * HPWL (Eq. 1) and overflow after round r's placement, r = 0..n_rounds
 * (Algorithm 1 records one solution per round).  hpwl, overflow: host
 * [n_rounds + 1], nullable; *n_records (nullable) receives n_rounds + 1, and
 * with cap smaller than that only the first cap records are written.  EINVAL
 * before the first place_hybro call. */
int place_get_hybro_rounds(place_t *h, int32_t copy, double *hpwl, double *overflow,
                           int32_t cap, int32_t *n_records);

/* Measurement helper: run n_iters iterations like place_step, but launched
 * stage by stage (no graph) with CUDA events between the stages, and add the
 * device time of each stage in milliseconds to stage_ms (host
 * [PLACE_N_STAGES]).  Synchronises.  Stages: */
#define PLACE_STAGE_DENSITY 0  /* clear map, scatter, overflow/rho, stop test */
#define PLACE_STAGE_SPECTRAL 1 /* the four transform GEMMs of the Poisson solve */
#define PLACE_STAGE_WIRELENGTH 2 /* WA value and gradients summed per cell (Eq. 3) */
#define PLACE_STAGE_CELLGRAD 3 /* per-cell gradient, field gather, preconditioning */
#define PLACE_STAGE_UPDATE 4   /* preconditioner, step size, Nesterov update */
#define PLACE_N_STAGES 5
int place_step_timed(place_t *h, int32_t n_iters, float *stage_ms);

/* Measurement helper: the floor of the wirelength stage's memory traffic on
 * this netlist.  Times (CUDA events, after one warm-up launch) a kernel that
 * does only the memory operations the WA pass of Eq. 3 cannot avoid: per pin
 * the streamed pin_cell and offset reads, one random 8-byte position gather
 * and one random 64-bit reduction into the cell's gradient sum; per net the
 * net_ptr read.  *ms receives the mean time of one pass over every copy.
 * The gradient sums are cleared afterwards; the placement state is otherwise
 * untouched.  Synchronises. */
int place_measure_wa_floor(place_t *h, int32_t reps, float *ms);

/* The density scatter against its floor at the current positions (all
 * copies): *ms_scatter receives the mean device time of the scatter as an
 * iteration runs it (the way each copy's last density pass chose), and
 * *ms_floor that of a kernel that makes only the same loads (position and
 * size per movable cell) and one 64-bit reduction into each bin the cell
 * covers, none of the exact overlap arithmetic.  Both use the density map as
 * scratch and leave it cleared (the next density pass rebuilds it).
 * Synchronises. */
int place_measure_scatter_floor(place_t *h, int32_t reps, float *ms_scatter, float *ms_floor);

/* Failure-path check of the bounded device waits.  Runs the first
 * tensor-core GEMM stage of copy 0 once with its copy producer idle, so that
 * no tile ever arrives: the MMA issuer's and the epilogue's waits give up
 * after about a second each, the kernel frees its tensor memory and raises
 * the device error flag, and this call returns PLACE_ETIMEOUT (the expected
 * outcome) after clearing the flag.  Nothing hangs and the handle stays
 * usable; the next iteration recomputes every stage.  EINVAL on a handle
 * without the tensor-core path.  Synchronises; takes about two seconds. */
int place_test_wait_timeout(place_t *h);

/* Failure-path check of the index checks of the bounds-checking build
 * (place_info.bounds_checked): one thread tests the index n_cells against
 * the cell count, as a kernel would before a position gather, and touches
 * no memory with it.  The check fails, so this call returns PLACE_EINTERNAL
 * (the expected outcome) with the site and the index in place_last_error(),
 * and the flag is cleared.  EINVAL in the normal build, which has no index
 * checks.  Synchronises. */
int place_test_bounds_check(place_t *h);

/* Density map and overflow of a placement without any device allocation.
 *
 * The paper has no counterpart to this function: it serves callers that
 * cannot allocate device memory when they need the overflow, such as a host
 * framework whose memory pool owns all device memory during a step, a
 * real-time service that forbids allocation after start-up, or a callback
 * that must not trigger the device-wide synchronisation an allocation can
 * cause.  Its scratch (64-bit density map, reduction partials and the area
 * sum) is one fixed-size array inside the library's module; every GPU that
 * loads the library holds it (about 8 MB) until the process exits.
 *
 * Computes what place_eval_density() computes for a handle of the same
 * design: the movable-cell map M in units of 2^-2F and tau = sum_b max(0, M_b
 * - t (A_b - F_b)) / A_mov, for n_movable cells with lower-left corners x, y
 * and sizes w, h (device float arrays).  Sizes are quantised like positions,
 * W = rint(w 2^F), and A_mov is the exact sum of W H, as in place_create.
 * frac_bits is the resolution F (place_info.frac_bits of a handle of the
 * same design); fixed_map is the fixed-cell map (device int64 [nx*ny],
 * x-major; NULL: no fixed cells).  Outputs: *overflow (device double) and,
 * if map_out is not NULL, the map (device int64 [nx*ny]).  Work runs
 * asynchronously on `stream`.
 *
 * Errors on the host: PLACE_EINVAL for nx * ny > PLACE_NOALLOC_MAX_BINS, a
 * die origin or bin size that is not a multiple of 2^-F, or other malformed
 * arguments; PLACE_ERANGE when frac_bits is too fine for the die (extent
 * 2^F >= 2^30, the rule place_create uses to choose F).  On the device: a cell
 * whose quantised size falls outside [1, 2^31), or a total area of 2^62 units
 * or more, makes *overflow NaN (the map is then not meaningful).
 *
 * Sharing: all calls use the one scratch array and each call clears it
 * first; calls whose work overlaps on the GPU (different streams or host
 * threads) race on it and must be serialised.  The first call with a given
 * device current looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
#define PLACE_NOALLOC_MAX_BINS (1024 * 1024)
int place_overflow_noalloc(const float *x, const float *y, const float *w, const float *h,
                           int32_t n_movable, const place_die *die, const place_bins *bins,
                           int32_t frac_bits, const int64_t *fixed_map, double *overflow,
                           int64_t *map_out, void *stream);

/* Device memory place_create would take for this netlist, die, bins and
 * parameters (an upper bound; no device work).  Used for admission control.
 * die may be NULL when params has no filler cells (their count needs it). */
int place_estimate_device_bytes(const place_netlist *nl, const place_die *die,
                                const place_bins *bins, const place_params *params,
                                int64_t *bytes);

/* ---- job server: continuous batching of placement and restart jobs -------
 * Algorithm 1 runs a placement, then perturbed re-placements ("restarts") of
 * its result.  The server runs many such jobs of different designs on one GPU
 * at once.  Jobs are admitted once they have arrived, their parent (for a
 * restart) has finished, a slot is free and their device footprint
 * (place_estimate_device_bytes) fits the budget; later jobs that fit may pass
 * a head job that does not.  Each active job keeps its state on the device
 * and runs on its own stream, iters_per_tick iterations per scheduling step,
 * so the work of all active jobs overlaps on the GPU.  A finished job's
 * handle stays resident while restarts depend on it; the last restart to be
 * admitted adopts it.  Results are those of the same job run alone (the
 * kernels are deterministic). */
#define PLACE_JOB_PLACE 0   /* place from the netlist's x0/y0 until the stop test */
#define PLACE_JOB_RESTART 1 /* perturb the parent's result (op, p, seed), re-place */

typedef struct place_server place_server;

typedef struct place_job {
  int32_t kind;      /* PLACE_JOB_* */
  int32_t op;        /* restart: PLACE_SHUFFLE_* or PLACE_WIREMASK */
  float p;           /* restart: strength */
  int32_t pad;
  uint64_t seed;     /* restart: SplitMix64 seed */
  int64_t parent;    /* restart: id of an earlier job of the same design */
  double arrival_s;  /* not admitted before this many seconds into place_server_run */
  double max_seconds; /* > 0: wall-clock budget from admission; the job is stopped at the
                       * first chunk boundary past it (status PLACE_JOB_EXPIRED); 0: none */
} place_job;

/* place_job_result.status */
#define PLACE_JOB_FINISHED 0  /* stopped by its stop test or max_iters */
#define PLACE_JOB_CANCELLED 1 /* place_server_cancel (or its parent's); a job cancelled
                               * before admission has no positions: NaN HPWL, hash 0 */
#define PLACE_JOB_EXPIRED 2   /* ran past max_seconds */

typedef struct place_job_result {
  int64_t id;
  int32_t kind, iterations, converged, status; /* status: PLACE_JOB_* */
  double arrival_s, admit_s, done_s; /* seconds since place_server_run started */
  double hpwl, overflow;             /* exact FP64 HPWL (Eq. 1) and overflow at the end */
  int64_t device_bytes;
  uint64_t position_hash;            /* FNV-1a of the final x then y arrays */
} place_job_result;

/* hbm_budget: bytes of device memory the jobs' handles may hold at once (a
 * finished job's saved positions, 8 bytes per cell while restarts of it are
 * pending, are not counted); max_active: concurrent jobs (1 = one job at a
 * time, in arrival order). */
int place_server_create(int64_t hbm_budget, int32_t max_active, int32_t iters_per_tick,
                        place_server **out);

/* Queue a job.  The netlist arrays are borrowed until the job has finished
 * (the server does not copy them); params->n_copies is forced to 1 and
 * params->autotune to 0 (tuning at admission would add to the job's latency).  *id
 * receives the job id (submission order from 0).  PLACE_ENOMEM if the job
 * alone exceeds the budget. */
int place_server_submit(place_server *s, const place_netlist *nl, const place_die *die,
                        const place_bins *bins, const place_params *params, const place_job *job,
                        int64_t *id);

/* Run until every queued job has finished (or timeout_s > 0 elapses:
 * PLACE_ETIMEOUT).  *makespan_s (nullable) receives the wall time. */
int place_server_run(place_server *s, double timeout_s, double *makespan_s);

/* Cancel job `id`: a queued job is never admitted (nor are its restarts); an
 * active one stops at its next chunk boundary, its in-flight kernels left to
 * finish.  May be called from another thread while place_server_run runs (it
 * only sets a flag that the run loop reads). */
int place_server_cancel(place_server *s, int64_t id);

/* Results of the finished jobs in submission order; *n receives their count
 * (out may be NULL to query it). */
int place_server_results(place_server *s, place_job_result *out, int32_t cap, int32_t *n);

/* Peak device bytes held by jobs and peak number of active jobs. */
int place_server_stats(place_server *s, int64_t *peak_bytes, int32_t *peak_active);

int place_server_destroy(place_server *s);

const char *place_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HYBRO_PLACE_H */
