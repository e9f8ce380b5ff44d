// Internal declarations of the sm_103a placement library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/hybro_place.h"
#include "common.cuh"

namespace hp {

// NVTX range over a scope (header-only NVTX v3: a no-op unless a profiler
// such as ncu --nvtx is attached).  The C-ABI entry points mark themselves,
// so a capture can be filtered to one call or one Hybro round.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kThreads = 256;       // block size of the per-cell / per-bin kernels
constexpr int kRedThreads = 1024;   // block size of the per-copy reducers
constexpr int kMaxCellBlocks = 1216;  // per copy: 8 blocks per SM on 152 SMs

// Optimiser scalars of one copy, resident on the device.  Kernels of one
// iteration read and write these; the host only reads them back on demand.
struct CopyState {
  double lam;        // density weight lambda (Eq. 2)
  double alpha;      // step length of the current iteration
  double a;          // Nesterov momentum sequence a_k
  double a_next;
  double coef;       // (a_k - 1) / a_{k+1}
  double tau;        // overflow at the current reference point
  double tau_prev;   // overflow of the previous reference point (drives gamma)
  double hpwl;       // HPWL of the last WA pass (pin max - min, FP32 pins)
  double hpwl_prev;
  double wl;         // WA wirelength of the last pass (Eq. 2 first term)
  double gamma;      // gamma of the current iteration (Eq. 3)
  int k;             // iterations done since reset
  int converged;
  int stopped;
  int parity;        // selects the current / previous gradient buffer
  int err;
  int n_back;        // steps redone in a row (backtracking)
  int reject;        // 1: the update redoes the last step (backtracking)
  int n_back_total;  // steps redone since reset
  double n_eff;      // effective number of occupied bins of the last density
                     // pass, (sum M)^2 / sum M^2; 0 before the first pass
  int n_hist;        // iteration records written since reset
  int pad_;
};

// Reduction slots (FP64) per copy: each kernel that reduces writes one value
// per block into its slot range; a reducer sums them in a fixed order.
enum Slot { S_TAU = 0, S_HPWL, S_WL, S_GW1, S_GD1, S_DG2, S_DV2, S_G2, S_HP64, S_COUNT };

// Last-block counters per copy.
enum Counter { C_FINISH = 0, C_CELL, C_PRE0, C_UPDATE, C_COUNT };

// The density scatter's ways of adding overlaps to the map (density.cu).
enum ScatterMode { SCAT_MERGED = 0, SCAT_TABLE = 1, SCAT_DIRECT = 2 };

// What the density-finish kernel does with the overflow it reduces.
enum FinishMode { FIN_ITER = 0, FIN_EVAL = 1, FIN_RESET = 2 };

struct Dev {
  // sizes.  With filler cells the library's cell order is [movable | fillers |
  // fixed]: n_mov counts the optimiser's cells (movable and fillers), n_real
  // the design's movable cells, n_fill the fillers, and n_cells all three.
  int K, n_cells, n_mov, n_nets, n_pins, nx, ny, G;
  int n_real, n_fill;
  int Gm;                     // per-copy stride of M: G, or 2 G with fillers
                              // (the fillers' map follows the movable one)
  int F;
  float gq, giq;              // 2^Fg, 2^-Fg: fixed-point scale of the WA gradient sums
  long long XL, YL, BW, BH;   // fixed point
  float scale;                // 2^F
  float inv_area_q;           // 2^-2F as float
  double t;                   // target density (float widened)
  long long t_mant;           // t = t_mant * 2^-t_shift exactly
  int t_shift;
  unsigned long long tA_lo, tA_hi;  // t_mant * A_bin as a 128-bit integer
  unsigned long long tA_floor;      // floor(t_mant * A_bin / 2^t_shift): a bin
                                    // without fixed cells overflows iff M > this
  double abin_q;              // BW * BH
  double mov_area_q;          // the design's movable area (units of 2^-2F): tau's denominator
  double fill_area_q;         // the fillers' area (units of 2^-2F)
  double die_xl, die_yl, die_xh, die_yh;
  float fxl, fyl, fxh, fyh;
  float fbw, fbh, fibw, fibh;  // bin width/height and their inverses (FP32)
  int BW32, BH32;             // BW, BH (below 2^26: nx, ny >= 16 and nx BW < 2^30)
  float ibw_q, ibh_q;         // 1 / BW, 1 / BH
  double w_bin, dref;
  int nb_red;                 // partial slots per reduction per copy
  int cell_blocks;            // blocks per copy for per-cell kernels
  int cg_blocks;              // blocks per copy of the cell-gradient kernel (one wave)
  int sms;                    // SMs of the device
  int bin_blocks;             // blocks per copy for per-bin kernels
  place_params prm;

  // netlist (library order: nets grouped by degree class)
  int *net_ptr;      // [n_nets+1]
  int *pin_cell;     // [n_pins]
  float2 *pin_off;   // [n_pins]
  float *net_w;      // [n_nets] or nullptr
  int has_net_w;
  float *w, *h;      // [n_cells]
  float2 *wh;        // [n_cells] (w, h) interleaved, for the per-cell optimiser kernels
  int *Wq, *Hq;      // [n_cells] quantised sizes
  float2 *pa;        // [n_mov] (pin count, charge area) per movable cell: the preconditioner's terms
  unsigned char *is_macro;  // [n_cells]
  // density stretching (null when off): per movable cell {x shift, y shift,
  // stretched W, stretched H} in fixed point, the density scale R (2^31 = 1),
  // and the stretched map that drives the field
  int4 *st;                  // [n_mov]
  unsigned int *sR;          // [n_mov]
  unsigned long long *Ms;    // [K][G]
  float inv_scale;           // 2^-F

  // per-copy state
  float2 *xy;                // [K][n_cells] reference positions v, interleaved (fixed part replicated)
  // per-cell (x, y) pairs are interleaved: one 8-byte access per cell
  float2 *u;                 // [K][n_mov] u_k
  float2 *vp;                // [K][n_mov] v_{k-1}
  float2 *g[2];              // [K][n_mov] preconditioned gradient, by parity
  float *gwx, *gwy, *gdx, *gdy;  // [K][n_mov] raw gradients
  float2 *up;                // [K][n_mov] u_k of the last accepted step (backtracking only)
  unsigned long long *gacc;  // [K][n_mov] WA gradient sums, two int32 fixed-point
                             // values packed as y * 2^32 + x (see add_pin_grad)
  unsigned long long *M;     // [K][Gm]: movable-cell map, then (fillers) the fillers' map
  long long *Fmap;           // [G]
  float *rho;                // [K][G]
  float *T;                  // [K][3][G] transform intermediates
  float *SB;                 // [K][3][G] spectral coefficients (x, y, psi)
  float *E;                  // [K][3][G] Ex, Ey, psi
  CopyState *cs;             // [K]
  double *part;              // [K][S_COUNT][nb_red]
  double *scal;              // [K][S_COUNT] reduced values (eval reductions)
  unsigned long long *tau_part;  // [K][nb_red][2] exact 128-bit overflow partials
  unsigned int *ctr;         // [K][C_COUNT] last-block counters
  float *conc_part;          // [K][nb_red] per-block sums of (M / A_bin)^2

  // spectral tables
  float *Cn, *Cm, *CTn, *STn, *STm, *CTm;  // transform matrices
  float *wu, *wv;                          // wavenumbers
  float *cu, *cv;                          // c_k / n factors

  // tensor-core spectral path (BF16x3): split operands, host tensor maps
  int tc;
  __nv_bfloat16 *rho_h, *rho_l;     // [K][G]
  __nv_bfloat16 *T_h, *T_l;         // [K][3][G]
  __nv_bfloat16 *SB_h, *SB_l;       // [K][3][G]
  __nv_bfloat16 *A1h, *A1l, *A2h, *A2l, *A3h, *A3l, *A4h, *A4l;
  int bfly;                         // the even/odd split of every transform (spectral.cu)
  float *wu_p, *wv_p, *cu_p, *cv_p; // with it: wu, wv, cu, cv in the frequency order of the
                                    // split (the even frequencies, then the odd ones)
  const void *tcm;                  // host array of 16 CUtensorMap (4 per GEMM stage)
  int tc_bn[4];                     // tile width N (64 or 128) of each GEMM stage
  int tc_split[4];                  // 1, or 2: split-K over two CTAs (tile width 128 only)
  int tc_split_ok[4];               // the stage has few enough tiles for split-K
  float *tc_ws;                     // split-K partial halves (stages with tc_split_ok)
  unsigned int *tc_ws_ctr;          // split-K arrivals per tile
  int tc_ws_tiles;                  // tiles the split-K workspace holds
  int *err;                         // [4]: bounded waits gave up; measurement sink; failed
                                    // index check (site, index) of the bounds-checking build

  // Hybro best solutions
  float2 *bxy;               // [K][n_cells]

  // per-iteration records, a ring of hist_cap per copy (place_get_history)
  place_iter_record *hist;   // [K][hist_cap]
  int hist_cap;

  // perturbation scratch
  unsigned long long *sort_key;  // [2^ceil(log2 n_cells)]
  unsigned int *sort_idx;
  unsigned int *sel_idx;          // [pow2]
  float *px_tmp, *py_tmp;         // [n_cells]
  int sort_n;                      // padded length

  // WA launch plan: nets [cls_begin[c], cls_begin[c+1]) belong to class c
  int cls_begin[8];
  int cls_split[8];           // the group classes' second sub-range (nets on more lanes)
  int n_cls;
  int wa_blocks[8];           // blocks per class per copy
  int wa_block_base[8];       // slot offset of the class's blocks
  int wa_blocks_total;
  int wa_big_cap;             // pins of a > 256-pin net kept in shared memory
  int wa_streams;             // graph branches of the WA classes (1..3, wa_branch_of)
  // density scatter: SCAT_MERGED below n_eff scat_t1, SCAT_TABLE below scat_t2,
  // SCAT_DIRECT above; scat_force >= 0 forces one way (tuning)
  double scat_t1, scat_t2;
  int scat_force;
};

// WireMask tables (built at create) and scratch (allocated on first use).
struct WmDev {
  int n_macros;         // movable macros
  int n_fixed;          // fixed cells: the obstacles every macro avoids
  int max_nets;         // most nets on one macro (at least 1)
  int nblk;             // candidate blocks per copy
  const int *order;     // [n_macros] macros by decreasing area, ties by index
  const int *mptr;      // [n_macros + 1] macro t's nets: mnet[mptr[t] .. mptr[t+1])
  const int *mnet;      // library net indices, in netlist order per macro
  const int *obst;      // [n_fixed + n_macros] fixed cells, then `order`
  double *box;          // [K][max_nets][8] per-net extents of the current macro
  double *fx, *fy;      // [K][nx], [K][ny] wire-mask axes
  double *bobj, *bdist; // [K][nblk] per-block winners
  int *bidx;            // [K][nblk]
};

// WA gradient sums per movable cell.  Each pin adds its (gx, gy), rounded to
// the fixed-point grid 2^-Fg, to its cell as the one 64-bit integer
// qy * 2^32 + qx.  Integer addition is exact and independent of order, so the
// sums are deterministic.  The create-time choice of Fg bounds every cell's
// |sum qx| and |sum qy| below 2^31; then the 64-bit total S equals
// (sum qy) 2^32 + sum qx exactly, its low 32 bits read as a signed integer
// are sum qx, and (S - sum qx) / 2^32 is sum qy.
__device__ __forceinline__ void add_pin_grad(const Dev &d, unsigned long long *acc, int cell,
                                             float gx, float gy) {
  if (cell >= d.n_mov) return;  // fixed cells take no gradient
  if (!HP_IN(d.err, cell, d.n_mov, BS_GRAD_CELL)) return;
  const long long qx = __float2int_rn(gx * d.gq), qy = __float2int_rn(gy * d.gq);
  atomicAdd(acc + cell, (unsigned long long)(qy * 4294967296LL + qx));
}
__device__ __forceinline__ float2 unpack_grad(const Dev &d, unsigned long long s) {
  const long long lo = (long long)(int)(unsigned int)(s & 0xffffffffull);
  const long long hi = ((long long)s - lo) / 4294967296LL;
  return make_float2((float)lo * d.giq, (float)hi * d.giq);
}

// ---- launchers (all enqueue on `st`) ------------------------------------
// eval != 0 ignores the stopped flag of the copy (stage-level evaluation).
// Programmatic dependent launch.  launch_pdl lets a kernel be scheduled
// while the kernel before it in the same stream drains; the kernel calls
// pdl_wait() before its first access to memory, which returns once that
// predecessor has completed and its writes are visible (for a kernel
// launched normally it returns at once).  Results are those of plain stream
// order; only the launch latency overlaps.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline void launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

void launch_scatter(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st);
void launch_scatter_fixed(const Dev &d, const float2 *xy, int n0, int n1,
                          unsigned long long *out, cudaStream_t st);
void launch_pack_xy(float2 *dst, const float *x, const float *y, int n, cudaStream_t st);
void launch_unpack_xy(float *x, float *y, const float2 *src, int n, cudaStream_t st);
void launch_density_finish(const Dev &d, int copy0, int ncopy, int mode, cudaStream_t st);
void launch_spectral(const Dev &d, int copy0, int ncopy, int with_psi, int eval, cudaStream_t st);
void launch_spectral_tc_stalled(const Dev &d, cudaStream_t st);
void launch_test_bounds(const Dev &d, cudaStream_t st);
void launch_wa(const Dev &d, int copy0, int ncopy, int eval, const float *gamma_override,
               cudaStream_t st);
// The WA classes of an iteration on d.wa_streams branches: branch b's classes
// run in sequence on st[b] (st[0..wa_streams-1]); every branch must already
// follow the positions' producer.
void launch_wa_branches(const Dev &d, int copy0, int ncopy, const cudaStream_t *st);
constexpr int kMaxWaStreams = 3;
void launch_hpwl64(const Dev &d, int copy0, int ncopy, cudaStream_t st);
int wa_prepare(int cap);
void launch_wa_floor(const Dev &d, int copy0, int ncopy, cudaStream_t st);
void launch_wa_class(const Dev &d, int cls, int copy0, int ncopy, int eval, cudaStream_t st);
void launch_scatter_main(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st);
void launch_scatter_floor(const Dev &d, int copy0, int ncopy, cudaStream_t st);

// Create-time tuning (autotune.cu).  Chooses, for the knobs the caller left
// automatic, the tensor-core GEMM tile width, the big-net shared-memory cap
// and the scatter's thresholds, by timing candidates on the handle's own
// device state.  The positions and optimiser state of every copy are
// overwritten; the caller restores them and drops any captured graph.
struct TuneOut {
  int bn[4];
  int split[4];
  int cap;
  int wa_streams;
  double t1, t2;
  double ms;     // host time spent
  int cached;    // 1: taken from the process-wide cache
};
struct TuneHooks {
  int (*encode_maps)(void *ctx);        // tensor maps for d.tc_bn
  float (*time_iters)(void *ctx, int n);  // ms per graph iteration from the start state
  void *ctx;
};
int autotune(Dev &d, int max_deg, cudaStream_t st, const TuneHooks &hk, TuneOut *out);
int cell_grad_blocks_per_sm();
void launch_cell_grad(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st);
void launch_precond0(const Dev &d, int copy0, int ncopy, cudaStream_t st);
void launch_update(const Dev &d, int copy0, int ncopy, cudaStream_t st);
void launch_reset(const Dev &d, int copy0, int ncopy, cudaStream_t st);
void launch_reduce_slot(const Dev &d, int slot, int nvals, int copy0, int ncopy, cudaStream_t st);
int launch_shuffle(const Dev &d, int copy, int op, float p, uint64_t seed, cudaStream_t st);
void launch_shuffle_finish(const Dev &d, int copy, int kcount, cudaStream_t st);
int wm_select_blocks(int G);
void launch_wiremask(const Dev &d, const WmDev &w, const int *mptr_host, int copy0, int ncopy,
                     cudaStream_t st);

// hooks for the job server (api.cu)
int step_async(place_t *h, int n, int *stopped_host, cudaEvent_t ev);
int copy_positions(place_t *dst, place_t *src, cudaEvent_t src_done);
cudaStream_t handle_stream(place_t *h);
int save_xy(place_t *h, float2 *dst);
int load_xy(place_t *h, const float2 *src);

// gamma of the weighted-average model from the previous overflow (Eq. 3)
__device__ __forceinline__ double gamma_of(const Dev &d, double tau_prev) {
  if (d.prm.constant_gamma > 0.f) return (double)d.prm.constant_gamma;
  return (double)d.prm.gamma_base * d.w_bin * pow(10.0, (20.0 / 9.0) * tau_prev - 11.0 / 9.0);
}

}  // namespace hp
