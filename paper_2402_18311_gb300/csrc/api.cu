// Host side of the C ABI declared in include/hybro_place.h: validation,
// netlist preprocessing, device-state layout, CUDA-graph iteration, stage
// evaluation and the Hybro driver (Algorithm 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <utility>
#include <vector>

#include "internal.cuh"
#include "spectral_tc.cuh"

using namespace hp;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(PLACE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

#define CKL()                                                                         \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess)                                                            \
      return fail(PLACE_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e_));   \
  } while (0)

// Bump allocator over one device allocation (256-byte aligned sub-arrays).
struct Arena {
  char *base = nullptr;
  size_t off = 0;
  template <typename T>
  T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += n * sizeof(T);
    return p;
  }
};

// WA launch classes: thread per net (<= 4 pins), 4-lane groups (<= 16),
// 16-lane groups (<= 64), warps (<= 256), a block per net (> 256); chunk
// sizes keep a chunk's pins within the staging buffers.
int degree_class(int deg) {
  if (deg <= 4) return 0;
  if (deg <= 16) return 1;
  if (deg <= 64) return 2;
  if (deg <= 256) return 3;
  return 4;
}
constexpr int kNetsPerBlock[4] = {256, 64, 16, 8};
// degree up to which a group class's net runs on half its lanes (4-lane class:
// 2 lanes for up to 8 pins; 16-lane class: 8 lanes for up to 32 pins; the
// warp class is not split)
constexpr int kGroupHalfDeg[4] = {0, 8, 32, 256};
// pins of a big net kept in shared memory: 3072 (24 KB) is the most that
// still lets eight 256-thread blocks share an SM; longer nets re-gather the rest
constexpr int kBigCapMax = 3072;
// the scatter's fixed-rule thresholds on the effective number of occupied
// bins: merged below the first, the shared table below the second, direct
// atomics above (the autotuner replaces them by measured crossovers)
constexpr double kScatterMergedBelow = 32.0;
constexpr double kScatterTableBelow = 1024.0;
constexpr int kMaxBigNetBlocks = 8192;  // one block per net above 256 pins, up to this many

bool is_integer(double v) { return std::floor(v) == v && std::isfinite(v); }

// Fixed-point resolution: the largest F <= 24 with max(|coordinate|, die
// width, die height) 2^F < 2^30 and total area 2^2F < 2^62 (the extent bound
// keeps bin-relative coordinates in int32); -1 when none fits.
int choose_frac_bits(const place_die *die, double total_area) {
  const double ext = std::max(std::max(std::max(std::fabs(die->xl), std::fabs(die->xh)),
                                       std::max(std::fabs(die->yl), std::fabs(die->yh))),
                              std::max(die->xh - die->xl, die->yh - die->yl));
  for (int f = 24; f >= 0; --f)
    if (ext * std::ldexp(1.0, f) < std::ldexp(1.0, 30) &&
        total_area * std::ldexp(1.0, 2 * f) < std::ldexp(1.0, 62))
      return f;
  return -1;
}

// Filler cells (ePlace's whitespace fillers, the density of Eq. 2): pinless
// movable cells that take up the whitespace the target density leaves.
//  * size: the mean quantised width and height of the movable non-macro
//    cells, each rounded to the nearest multiple of 2^-F (ties to even);
//  * count: floor(max(0, t (A_die - A_fixed) - A_mov) / (w_f h_f)), with
//    A_fixed the fixed cells' area inside the die (exact in fixed point) and
//    A_mov the movable cells' quantised area, in float64 in that order;
//  * start: filler j at (xl + u (xh - xl - w_f), yl + v (yh - yl - h_f))
//    rounded to float32, u and v the (2j+1)-th and (2j+2)-th SplitMix64
//    outputs from kFillerSeed as (z >> 11) 2^-53.
constexpr unsigned long long kFillerSeed = 0x46494C4C45525321ull;  // "FILLERS!"
struct FillPlan {
  int Wf = 0, Hf = 0;   // size in units of 2^-F
  long long n = 0;      // count
};

FillPlan plan_fillers(const place_netlist *nl, const place_die *die, const place_bins *bins,
                      int F, unsigned __int128 mov_area_q) {
  FillPlan fp;
  const double s = std::ldexp(1.0, F);
  const int Mv = nl->n_movable, C = nl->n_cells;
  long long sw = 0, sh = 0, cnt = 0;
  for (int i = 0; i < Mv; ++i) {
    if (nl->is_macro && nl->is_macro[i]) continue;
    sw += (long long)std::nearbyint((double)nl->w[i] * s);
    sh += (long long)std::nearbyint((double)nl->h[i] * s);
    ++cnt;
  }
  if (cnt == 0) return fp;
  fp.Wf = std::max(1, (int)std::nearbyint((double)sw / (double)cnt));
  fp.Hf = std::max(1, (int)std::nearbyint((double)sh / (double)cnt));
  // fixed area inside the die: each fixed rectangle clipped to the die
  const long long XL = (long long)(die->xl * s), YL = (long long)(die->yl * s);
  const long long XH = XL + (long long)std::nearbyint((die->xh - die->xl) * s);
  const long long YH = YL + (long long)std::nearbyint((die->yh - die->yl) * s);
  unsigned __int128 fixed_q = 0;
  for (int i = Mv; i < C; ++i) {
    const long long X = (long long)std::nearbyint((double)nl->x0[i] * s);
    const long long Y = (long long)std::nearbyint((double)nl->y0[i] * s);
    const long long W = (long long)std::nearbyint((double)nl->w[i] * s);
    const long long H = (long long)std::nearbyint((double)nl->h[i] * s);
    const long long ox = std::min(X + W, XH) - std::max(X, XL);
    const long long oy = std::min(Y + H, YH) - std::max(Y, YL);
    if (ox > 0 && oy > 0) fixed_q += (unsigned __int128)ox * (unsigned __int128)oy;
  }
  const double s2 = std::ldexp(1.0, -2 * F);
  const double a_die = (die->xh - die->xl) * (die->yh - die->yl);
  const double fill = (double)bins->target_density * (a_die - (double)fixed_q * s2) -
                      (double)mov_area_q * s2;
  const double wf = fp.Wf * std::ldexp(1.0, -F), hf = fp.Hf * std::ldexp(1.0, -F);
  fp.n = fill > 0.0 ? (long long)std::floor(fill / (wf * hf)) : 0;
  return fp;
}

void filler_start(long long n, const place_die *die, double wf, double hf, float2 *out) {
  auto splitmix = [](unsigned long long k) {  // (k+1)-th output from kFillerSeed
    unsigned long long z = kFillerSeed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (long long j = 0; j < n; ++j) {
    const double u = (double)(splitmix(2 * j) >> 11) * std::ldexp(1.0, -53);
    const double v = (double)(splitmix(2 * j + 1) >> 11) * std::ldexp(1.0, -53);
    out[j] = make_float2((float)(die->xl + u * ((die->xh - die->xl) - wf)),
                         (float)(die->yl + v * ((die->yh - die->yl) - hf)));
  }
}

// PLACE_DCT_AUTO: the tensor-core path wherever the grid allows it.
int resolve_dct_mode(int mode, int nx, int ny) {
  if (mode != PLACE_DCT_AUTO) return mode;
  return (nx % 128 == 0 && ny % 128 == 0) ? PLACE_DCT_BF16X3 : PLACE_DCT_FP32;
}

// The even/odd split of the tensor-core solve: each half of a side must
// hold whole 128-row tiles (and each half of a contraction whole pairs of
// 64-element K-blocks), so both sides are multiples of 256.
int use_fold(int tc, int fold, int nx, int ny) {
  return (tc && fold && nx % 256 == 0 && ny % 256 == 0) ? 1 : 0;
}

}  // namespace

namespace hp {
// Lets other translation units report through place_last_error().
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace hp

struct place_t {
  Dev d{};
  cudaStream_t stream = nullptr;     // caller's stream
  cudaStream_t cap = nullptr;        // private stream used for graph capture
  cudaStream_t cap2 = nullptr;       // captured streams of the wirelength branches
  cudaStream_t cap3 = nullptr, cap4 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_join2 = nullptr, ev_join3 = nullptr;
  void *mem = nullptr;
  size_t mem_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the same iteration with the k = 0 preconditioning pass (k_precond0),
  // launched for the first iteration after a reset of any copy; `exec`
  // leaves that pass out, where it would only find every copy past k = 0
  cudaGraph_t graph0 = nullptr;
  cudaGraphExec_t exec0 = nullptr;
  bool k0_pending = true;
  CUtensorMap maps[16];              // tensor maps of the tcgen05 spectral path
  int n_cand_all = 0, n_cand_macro = 0;
  // WireMask: host tables built at create, device copy made on first use
  std::vector<int> wm_order, wm_ptr, wm_net, wm_obst;
  int wm_max_nets = 1;
  void *wm_mem = nullptr;
  WmDev wm{};
  // one captured graph per (first copy, copies) of a WireMask pass: the pass
  // is four small kernels per macro, so its launches dominate otherwise
  std::map<std::pair<int, int>, cudaGraphExec_t> wm_graphs;
  // Hybro bookkeeping (host)
  std::vector<double> best_hpwl, best_tau;
  std::vector<int> best_round;
  std::vector<double> round_hpwl, round_tau;  // [K][rounds] of the last place_hybro
  int n_round_records = 0;
  int autotuned = 0;
  double autotune_ms = 0.0;
};

extern "C" {

const char *place_last_error(void) { return g_err.c_str(); }

void place_default_params(place_params *p) {
  if (!p) return;
  p->n_copies = 1;
  p->gamma_base = 4.0f;
  p->lambda_eta = 1e-3f;
  p->alpha0 = 0.05f;
  p->hpwl_ref = 0.3f;
  p->mu_base = 1.1f;
  p->mu_lo = 0.95f;
  p->mu_hi = 1.05f;
  p->tau_stop = 0.07f;
  p->max_iters = 1000;
  p->constant_gamma = 0.0f;
  p->dct_mode = PLACE_DCT_AUTO;
  p->max_backtracks = 0;
  p->stretch = 0;
  p->autotune = 1;
  p->scatter_mode = -1;
  p->gemm_bn = 0;
  p->wa_big_cap = 0;
  p->gemm_split = 0;
  p->wa_streams = 0;
  p->fillers = 0;
  p->macro_precond = 1.0f;
  p->dct_fold = 1;
}

int place_destroy(place_t *h) {
  if (!h) return PLACE_OK;
  cudaStreamSynchronize(h->stream);  // no work of this handle may still run
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->exec0) cudaGraphExecDestroy(h->exec0);
  if (h->graph0) cudaGraphDestroy(h->graph0);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->cap2) cudaStreamDestroy(h->cap2);
  if (h->cap3) cudaStreamDestroy(h->cap3);
  if (h->cap4) cudaStreamDestroy(h->cap4);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_join2) cudaEventDestroy(h->ev_join2);
  if (h->ev_join3) cudaEventDestroy(h->ev_join3);
  if (h->mem) cudaFreeAsync(h->mem, h->stream);  // stream-ordered: no device-wide sync
  for (auto &g : h->wm_graphs) cudaGraphExecDestroy(g.second);
  if (h->wm_mem) cudaFreeAsync(h->wm_mem, h->stream);
  delete h;
  return PLACE_OK;
}

}  // extern "C"

namespace {

// Device layout of every array the handle owns.
void layout(Dev &d, Arena &a, int n_copies) {
  const size_t K = n_copies, C = d.n_cells, Mv = d.n_mov, P = d.n_pins, G = d.G;
  d.net_ptr = a.take<int>(d.n_nets + 1);
  d.net_w = d.has_net_w ? a.take<float>(std::max(d.n_nets, 1)) : nullptr;
  d.pin_cell = a.take<int>(P);
  d.pin_off = a.take<float2>(P);
  d.w = a.take<float>(C);
  d.h = a.take<float>(C);
  d.wh = a.take<float2>(C);
  d.Wq = a.take<int>(C);
  d.Hq = a.take<int>(C);
  d.pa = a.take<float2>(Mv);
  d.is_macro = a.take<unsigned char>(C);
  d.st = d.prm.stretch ? a.take<int4>(std::max<size_t>(Mv, 1)) : nullptr;
  d.sR = d.prm.stretch ? a.take<unsigned int>(std::max<size_t>(Mv, 1)) : nullptr;
  d.Ms = d.prm.stretch ? a.take<unsigned long long>(K * G) : nullptr;
  d.xy = a.take<float2>(K * C);
  d.u = a.take<float2>(K * Mv);
  // v_{k-1} is kept only for backtracking (the redone step starts there);
  // otherwise k_update reduces |v_{k+1} - v_k| itself
  d.vp = d.prm.max_backtracks > 0 ? a.take<float2>(K * Mv) : nullptr;
  for (int q = 0; q < 2; ++q) d.g[q] = a.take<float2>(K * Mv);
  d.gwx = a.take<float>(K * Mv);
  d.gwy = a.take<float>(K * Mv);
  d.gdx = a.take<float>(K * Mv);
  d.gdy = a.take<float>(K * Mv);
  d.up = d.prm.max_backtracks > 0 ? a.take<float2>(K * Mv) : nullptr;
  d.gacc = a.take<unsigned long long>(K * std::max<size_t>(Mv, 1));
  d.M = a.take<unsigned long long>(K * (size_t)d.Gm);
  d.Fmap = a.take<long long>(G);
  d.rho = a.take<float>(K * G);
  d.T = a.take<float>(K * 3 * G);
  d.SB = a.take<float>(K * 3 * G);
  d.E = a.take<float>(K * 3 * G);
  d.cs = a.take<CopyState>(K);
  d.hist_cap = PLACE_HISTORY_CAP;
  d.hist = a.take<place_iter_record>(K * (size_t)d.hist_cap);
  d.part = a.take<double>(K * S_COUNT * (size_t)d.nb_red);
  d.scal = a.take<double>(K * S_COUNT);
  d.tau_part = a.take<unsigned long long>(K * 2 * (size_t)d.nb_red);
  d.ctr = a.take<unsigned int>(K * C_COUNT);
  d.conc_part = a.take<float>(K * (size_t)d.nb_red);
  d.Cn = a.take<float>((size_t)d.ny * d.ny);
  d.CTn = a.take<float>((size_t)d.ny * d.ny);
  d.STn = a.take<float>((size_t)d.ny * d.ny);
  d.Cm = a.take<float>((size_t)d.nx * d.nx);
  d.CTm = a.take<float>((size_t)d.nx * d.nx);
  d.STm = a.take<float>((size_t)d.nx * d.nx);
  d.wu = a.take<float>(d.nx);
  d.wv = a.take<float>(d.ny);
  d.cu = a.take<float>(d.nx);
  d.cv = a.take<float>(d.ny);
  d.bxy = a.take<float2>(K * C);
  d.sort_key = a.take<unsigned long long>(d.sort_n);
  d.sort_idx = a.take<unsigned int>(d.sort_n);
  d.sel_idx = a.take<unsigned int>(d.sort_n);
  d.px_tmp = a.take<float>(C);
  d.py_tmp = a.take<float>(C);
  d.err = a.take<int>(4);  // [0]: bounded waits gave up; [1]: a sink for measurement kernels;
                           // [2], [3]: a failed index check (bounds-checking build)
  if (d.tc) {
    const size_t nx2 = (size_t)d.nx * d.nx, ny2 = (size_t)d.ny * d.ny;
    d.rho_h = a.take<__nv_bfloat16>(K * G);
    d.rho_l = a.take<__nv_bfloat16>(K * G);
    d.T_h = a.take<__nv_bfloat16>(K * 3 * G);
    d.T_l = a.take<__nv_bfloat16>(K * 3 * G);
    d.SB_h = a.take<__nv_bfloat16>(K * G);
    d.SB_l = a.take<__nv_bfloat16>(K * G);
    d.A1h = a.take<__nv_bfloat16>(ny2);
    d.A1l = a.take<__nv_bfloat16>(ny2);
    d.A2h = a.take<__nv_bfloat16>(nx2);
    d.A2l = a.take<__nv_bfloat16>(nx2);
    d.A3h = a.take<__nv_bfloat16>(3 * ny2);
    d.A3l = a.take<__nv_bfloat16>(3 * ny2);
    d.A4h = a.take<__nv_bfloat16>(3 * nx2);
    d.A4l = a.take<__nv_bfloat16>(3 * nx2);
    if (d.bfly) {
      d.wu_p = a.take<float>(d.nx);
      d.cu_p = a.take<float>(d.nx);
      d.wv_p = a.take<float>(d.ny);
      d.cv_p = a.take<float>(d.ny);
    }
    // split-K workspace: two 128 x 128 FP32 halves per tile of the largest
    // stage that may split (a stage with at most half as many 128-wide tiles
    // as the device has SMs)
    const int sms = d.sms > 0 ? d.sms : 152;
    const size_t t1 = (size_t)(d.nx / 128) * (d.ny / 128) * K;
    // the inverse stages have two fields; with the even/odd split they
    // cover half the rows of each
    const size_t t3 = d.bfly ? t1 : 2 * t1;
    const size_t tiles[4] = {t1, t1, t3, t3};
    size_t ws_tiles = 0;
    for (int s = 0; s < 4; ++s) {
      d.tc_split_ok[s] = 2 * tiles[s] <= (size_t)sms ? 1 : 0;
      if (d.tc_split_ok[s]) ws_tiles = std::max(ws_tiles, tiles[s]);
    }
    d.tc_ws_tiles = (int)ws_tiles;
    d.tc_ws = ws_tiles ? a.take<float>(ws_tiles * 2 * 128 * 128) : nullptr;
    d.tc_ws_ctr = ws_tiles ? a.take<unsigned int>(ws_tiles) : nullptr;
  }
}

int encode_tc_maps(place_t *h);

// Split the FP32 transform matrices into bf16 pairs and encode the tensor
// maps of the four GEMM stages.
int setup_tc(place_t *h) {
  Dev &d = h->d;
  cudaStream_t st = h->stream;
  const size_t nx2 = (size_t)d.nx * d.nx, ny2 = (size_t)d.ny * d.ny;
  if (!d.bfly) {  // the even/odd split's operands were built at create
  launch_split_bf16(d.Cn, d.A1h, d.A1l, ny2, st);
  launch_split_bf16(d.Cm, d.A2h, d.A2l, nx2, st);
  launch_split_bf16(d.CTn, d.A3h, d.A3l, ny2, st);
  // S_N with column v scaled by w_v: stage 3's y field from the one
  // coefficient field of stage 2
  launch_split_bf16_colscale(d.STn, d.wv, d.A3h + ny2, d.A3l + ny2, d.ny, d.ny, st);
  launch_split_bf16(d.CTn, d.A3h + 2 * ny2, d.A3l + 2 * ny2, ny2, st);
  launch_split_bf16(d.STm, d.A4h, d.A4l, nx2, st);
  launch_split_bf16(d.CTm, d.A4h + nx2, d.A4l + nx2, nx2, st);
  launch_split_bf16(d.CTm, d.A4h + 2 * nx2, d.A4l + 2 * nx2, nx2, st);
  }
  CKL();
  const int nx = d.nx, ny = d.ny, K = d.K;
  // tile width per stage, unless forced or tuned: 128; 64 only for grids so
  // small that 128-wide tiles would occupy under a quarter of the SMs
  const int sms = d.sms;
  const int t3 = (nx / 128) * (ny / 128) * (d.bfly ? 1 : 2) * K;  // two fields; half the rows
  const int tiles128[4] = {(nx / 128) * (ny / 128) * K, (ny / 128) * (nx / 128) * K, t3, t3};
  for (int s = 0; s < 4; ++s) {
    d.tc_bn[s] = d.prm.gemm_bn ? d.prm.gemm_bn : (tiles128[s] * 4 <= sms ? 64 : 128);
    d.tc_split[s] = (d.prm.gemm_split == 2 && d.tc_split_ok[s] && d.tc_bn[s] == 128) ? 2 : 1;
  }
  if (d.tc_ws_ctr) CK(cudaMemsetAsync(d.tc_ws_ctr, 0, sizeof(unsigned int) * d.tc_ws_tiles, h->stream));
  if (tc_prepare()) return fail(PLACE_ECUDA, "cannot reserve %d bytes of shared memory", tc_smem_bytes(128));
  return encode_tc_maps(h);
}

// Tensor maps of the four GEMM stages for the tile widths in d.tc_bn.
int encode_tc_maps(place_t *h) {
  Dev &d = h->d;
  const int nx = d.nx, ny = d.ny, K = d.K;
  // the even/odd split: forward A matrices with half the contraction,
  // inverse ones with half the rows, stage 1's B tile in two mirrored halves
  const int f = d.bfly ? 2 : 1;
  struct M { const void *p; int k, rows, batch, box; } spec[16] = {
      {d.A1h, ny / f, ny, 1, 128}, {d.A1l, ny / f, ny, 1, 128},
      {d.rho_h, ny, nx, K, d.tc_bn[0] / f}, {d.rho_l, ny, nx, K, d.tc_bn[0] / f},
      {d.A2h, nx / f, nx, 1, 128}, {d.A2l, nx / f, nx, 1, 128},
      {d.T_h, nx, ny, 3 * K, d.tc_bn[1]}, {d.T_l, nx, ny, 3 * K, d.tc_bn[1]},
      {d.A3h, ny, ny / f, 3, 128}, {d.A3l, ny, ny / f, 3, 128},
      {d.SB_h, ny, nx, K, d.tc_bn[2]}, {d.SB_l, ny, nx, K, d.tc_bn[2]},
      {d.A4h, nx, nx / f, 3, 128}, {d.A4l, nx, nx / f, 3, 128},
      {d.T_h, nx, ny, 3 * K, d.tc_bn[3]}, {d.T_l, nx, ny, 3 * K, d.tc_bn[3]}};
  for (int i = 0; i < 16; ++i) {
    int r = make_map_bf16_3d(&h->maps[i], spec[i].p, spec[i].k, spec[i].rows, spec[i].batch, spec[i].box);
    if (r) return fail(PLACE_ECUDA, "tensor map %d could not be encoded (%d)", i, r);
  }
  d.tcm = h->maps;
  return PLACE_OK;
}

// Context of the tuning hooks: the handle and the start positions.
struct TuneCtx {
  place_t *h;
  const float2 *xy0;
};

int encode_tc_maps_cb(void *ctx) { return encode_tc_maps(static_cast<TuneCtx *>(ctx)->h); }

void drop_graph(place_t *h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->exec0) cudaGraphExecDestroy(h->exec0);
  if (h->graph0) cudaGraphDestroy(h->graph0);
  h->exec = h->exec0 = nullptr;
  h->graph = h->graph0 = nullptr;
}

int enqueue_reset(place_t *h, int c0, int n);
int ensure_graph(place_t *h);
cudaError_t launch_iter(place_t *h);

// Every copy back at the start, a graph captured for the current device
// state, two warm-up iterations, then n timed ones: ms per iteration
// (negative on a CUDA error).
float time_iters_cb(void *ctx, int n) {
  TuneCtx *t = static_cast<TuneCtx *>(ctx);
  place_t *h = t->h;
  Dev &d = h->d;
  const size_t C = d.n_cells;
  for (int c = 0; c < d.K; ++c)
    if (cudaMemcpyAsync(d.xy + c * C, t->xy0, sizeof(float2) * C, cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
      return -1.f;
  if (enqueue_reset(h, 0, d.K)) return -1.f;
  drop_graph(h);
  if (ensure_graph(h)) return -1.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  for (int i = 0; i < 2; ++i) launch_iter(h);
  cudaEventRecord(e0, h->stream);
  for (int i = 0; i < n; ++i) launch_iter(h);
  cudaEventRecord(e1, h->stream);
  float ms = -1.f;
  if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
    ms /= n;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? ms : -1.f;
}

const char *bound_site_name(int site) {
  switch (site) {
    case BS_WA_PIN: return "WA: a net's pin range";
    case BS_WA_CELL: return "WA: a pin's cell";
    case BS_HPWL_PIN: return "HPWL: a net's pin range";
    case BS_HPWL_CELL: return "HPWL: a pin's cell";
    case BS_GRAD_CELL: return "WA: the cell of a pin gradient";
    case BS_MAP_BIN: return "density scatter: a map entry";
    case BS_FIELD_BIN: return "cell gradient: a field entry";
    case BS_TILE_ROW: return "tensor-core GEMM: an output row or column";
    case BS_WM_NET: return "WireMask: a net or pin";
    case BS_WM_CELL: return "WireMask: a cell";
    case BS_WM_BIN: return "WireMask: a bin";
    case BS_PERM: return "Shuffle: a permutation entry";
    default: return "unknown site";
  }
}

// Device-side error flags, call after a sync: [0] a bounded wait gave up;
// [2], [3] the first failed index check and its index (bounds-checking build
// only).  Reported flags are cleared.
int check_dev_err(place_t *h) {
  int e[4] = {0, 0, 0, 0};
  CK(cudaMemcpy(e, h->d.err, sizeof e, cudaMemcpyDeviceToHost));
  if (e[2]) {
    CK(cudaMemset(h->d.err + 2, 0, 2 * sizeof(int)));
    return fail(PLACE_EINTERNAL, "index check failed at %s (site %d), index %d", bound_site_name(e[2]),
                e[2], e[3]);
  }
  if (e[0]) return fail(PLACE_ETIMEOUT, "a device wait gave up (tensor-core pipeline)");
  return PLACE_OK;
}

// Optimiser reset of copies [c0, c0+n): clamp, u = v, scalars, tau_{-1}.
int enqueue_reset(place_t *h, int c0, int n) {
  Dev &d = h->d;
  cudaStream_t st = h->stream;
  h->k0_pending = true;  // the next iteration preconditions these copies' first step
  launch_reset(d, c0, n, st);
  CK(cudaMemsetAsync(d.M + (size_t)c0 * d.Gm, 0, sizeof(unsigned long long) * d.Gm * n, st));
  launch_scatter(d, c0, n, 1, st);
  launch_density_finish(d, c0, n, FIN_RESET, st);
  CKL();
  return PLACE_OK;
}

// One Nesterov iteration of every copy (the graph body).  The wirelength
// kernels depend only on the positions and on gamma_k (from the previous
// iteration's overflow), so they run on their own branches (d.wa_streams of
// them) beside the density scatter and the tensor-core Poisson solve, and
// join before the per-cell gradient.
void enqueue_iteration(const Dev &d, cudaStream_t st, const cudaStream_t *wst, cudaEvent_t fork,
                       const cudaEvent_t *join, bool with_precond0) {
  const int K = d.K;
  const int nb = std::max(1, std::min(d.wa_streams, kMaxWaStreams));
  cudaEventRecord(fork, st);
  for (int b = 0; b < nb; ++b) cudaStreamWaitEvent(wst[b], fork, 0);
  launch_wa_branches(d, 0, K, wst);
  for (int b = 0; b < nb; ++b) cudaEventRecord(join[b], wst[b]);
  cudaMemsetAsync(d.M, 0, sizeof(unsigned long long) * (size_t)d.Gm * K, st);
  launch_scatter(d, 0, K, 0, st);
  launch_density_finish(d, 0, K, FIN_ITER, st);
  launch_spectral(d, 0, K, 0, 0, st);
  for (int b = 0; b < nb; ++b) cudaStreamWaitEvent(st, join[b], 0);
  launch_cell_grad(d, 0, K, 0, st);
  if (with_precond0) launch_precond0(d, 0, K, st);
  launch_update(d, 0, K, st);
}

int ensure_graph(place_t *h) {
  if (h->exec && h->exec0) return PLACE_OK;
  drop_graph(h);
  const cudaStream_t wst[kMaxWaStreams] = {h->cap2, h->cap3, h->cap4};
  const cudaEvent_t joins[kMaxWaStreams] = {h->ev_join, h->ev_join2, h->ev_join3};
  for (int with0 = 0; with0 < 2; ++with0) {
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    enqueue_iteration(h->d, h->cap, wst, h->ev_fork, joins, with0 != 0);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess) return fail(PLACE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    (with0 ? h->graph0 : h->graph) = g;
    CK(cudaGraphInstantiate(with0 ? &h->exec0 : &h->exec, g, 0));
  }
  return PLACE_OK;
}

// One iteration of every copy: the graph with the k = 0 preconditioning pass
// when a reset since the last iteration may have left a copy at k = 0, the
// one without it otherwise (the two compute the same: the pass does nothing
// for a copy past k = 0).  ensure_graph must have succeeded.
cudaError_t launch_iter(place_t *h) {
  if (h->k0_pending) {
    h->k0_pending = false;
    return cudaGraphLaunch(h->exec0, h->stream);
  }
  return cudaGraphLaunch(h->exec, h->stream);
}

// Interleaved device positions -> caller's x, y (host or device) through the
// handle's scratch; synchronises.
int copy_out_xy(place_t *h, const float2 *src, float *x, float *y) {
  const Dev &d = h->d;
  const int C = d.n_cells - d.n_fill;  // the design's cells: movable, then fixed
  launch_unpack_xy(d.px_tmp, d.py_tmp, src, d.n_real, h->stream);
  launch_unpack_xy(d.px_tmp + d.n_real, d.py_tmp + d.n_real, src + d.n_mov, C - d.n_real, h->stream);
  CKL();
  if (x) CK(cudaMemcpyAsync(x, h->d.px_tmp, sizeof(float) * C, cudaMemcpyDefault, h->stream));
  if (y) CK(cudaMemcpyAsync(y, h->d.py_tmp, sizeof(float) * C, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PLACE_OK;
}

int check_copy(const place_t *h, int copy, bool allow_all) {
  if (!h) return fail(PLACE_EINVAL, "null handle");
  if (copy == -1 && allow_all) return PLACE_OK;
  if (copy < 0 || copy >= h->d.K) return fail(PLACE_EINVAL, "copy %d out of range [0,%d)", copy, h->d.K);
  return PLACE_OK;
}

// Device copy of the WireMask tables, and its scratch, made on the first
// WireMask call and freed with the handle (stream-ordered).
int ensure_wiremask(place_t *h) {
  if (h->wm_mem) return PLACE_OK;
  const Dev &d = h->d;
  WmDev &w = h->wm;
  w.n_macros = (int)h->wm_order.size();
  w.n_fixed = d.n_cells - d.n_mov;
  w.max_nets = h->wm_max_nets;
  w.nblk = wm_select_blocks(d.G);
  const size_t K = d.K;
  Arena a;
  int *order = nullptr, *mptr = nullptr, *mnet = nullptr, *obst = nullptr;
  auto lay = [&]() {
    order = a.take<int>(w.n_macros);
    mptr = a.take<int>(w.n_macros + 1);
    mnet = a.take<int>(std::max<size_t>(h->wm_net.size(), 1));
    obst = a.take<int>(h->wm_obst.size());
    w.box = a.take<double>(K * w.max_nets * 8);
    w.fx = a.take<double>(K * d.nx);
    w.fy = a.take<double>(K * d.ny);
    w.bobj = a.take<double>(K * w.nblk);
    w.bdist = a.take<double>(K * w.nblk);
    w.bidx = a.take<int>(K * w.nblk);
  };
  lay();
  void *mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, a.off + 256, h->stream);
  if (e != cudaSuccess)
    return fail(PLACE_ENOMEM, "WireMask scratch of %zu bytes: %s", a.off, cudaGetErrorString(e));
  h->wm_mem = mem;
  a = Arena();
  a.base = (char *)mem;
  lay();
  w.order = order; w.mptr = mptr; w.mnet = mnet; w.obst = obst;
  auto up = [&](int *dst, const std::vector<int> &src) -> int {
    if (!src.empty())
      CK(cudaMemcpyAsync(dst, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice, h->stream));
    return PLACE_OK;
  };
  int rc = up(order, h->wm_order);
  if (!rc) rc = up(mptr, h->wm_ptr);
  if (!rc) rc = up(mnet, h->wm_net);
  if (!rc) rc = up(obst, h->wm_obst);
  if (rc) {  // the next WireMask call starts over
    cudaFreeAsync(h->wm_mem, h->stream);
    h->wm_mem = nullptr;
  }
  return rc;
}

void host_dct_tables(int n, double h, std::vector<float> &C, std::vector<float> &CT,
                     std::vector<float> &S, std::vector<float> &ST, std::vector<float> &w,
                     std::vector<float> &c) {
  // C[k][i] = cos(pi k (i + 1/2) / n); CT = C^T; ST[i][k] = sin(pi k (i + 1/2) / n); S = ST^T
  C.assign((size_t)n * n, 0.f); CT = C; S = C; ST = C;
  w.assign(n, 0.f); c.assign(n, 0.f);
  for (int k = 0; k < n; ++k) {
    w[k] = (float)(M_PI * k / (n * h));
    c[k] = (float)((k == 0 ? 1.0 : 2.0) / n);
    for (int i = 0; i < n; ++i) {
      double arg = M_PI * k * (i + 0.5) / n;
      float cv = (float)std::cos(arg), sv = (float)std::sin(arg);
      C[(size_t)k * n + i] = cv;
      CT[(size_t)i * n + k] = cv;
      S[(size_t)k * n + i] = sv;
      ST[(size_t)i * n + k] = sv;
    }
  }
}

// Frequency order of the even/odd split: position p < n/2 holds frequency
// 2p, position n/2 + p frequency 2p + 1.
inline int fold_freq(int p, int n) { return p < n / 2 ? 2 * p : 2 * (p - n / 2) + 1; }

// FP32 -> bf16, rounding to nearest even (finite values), and the bf16 pair
// (hi, lo) of x with hi = bf16(x), lo = bf16(x - hi), as the device splits.
inline uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
inline void host_split(float v, uint16_t &hi, uint16_t &lo) {
  hi = host_bf16(v);
  const uint32_t hu = (uint32_t)hi << 16;
  float hf;
  std::memcpy(&hf, &hu, 4);
  lo = host_bf16(v - hf);
}

// The operands of the four stages with the even/odd split (the tensor
// maps' shapes in encode_tc_maps):
//   A1 [ny][ny/2]: row p = Cn row fold_freq(p), columns y < ny/2 (the forward
//     transform of rho's even/odd halves; the odd rows read the second half)
//   A2 [nx][nx/2]: the same for Cm
//   A3 [3][ny/2][ny]: rows y < ny/2 of the three inverse y matrices (CT,
//     S diag(w_v), CT), columns in the split frequency order
//   A4 [3][nx/2][nx]: rows x < nx/2 of S, CT, CT along x, the same order
// and wu, wv, cu, cv in that order.  Values are the FP32 tables' (the y
// field's products rounded once to FP32, as the device split does).
int upload_fold_tables(Dev &d, cudaStream_t st, const std::vector<float> &Cn,
                       const std::vector<float> &CTn, const std::vector<float> &STn,
                       const std::vector<float> &Cm, const std::vector<float> &CTm,
                       const std::vector<float> &STm, const std::vector<float> &wu,
                       const std::vector<float> &wv, const std::vector<float> &cu,
                       const std::vector<float> &cv) {
  const int nx = d.nx, ny = d.ny;
  std::vector<uint16_t> hi, lo;
  auto put = [&](__nv_bfloat16 *dh, __nv_bfloat16 *dl) -> int {
    if (cudaMemcpyAsync(dh, hi.data(), 2 * hi.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dl, lo.data(), 2 * lo.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(PLACE_ECUDA, "upload of the transform matrices failed");
    return PLACE_OK;
  };
  // forward: [n][n/2] rows in the split order
  auto fwd = [&](const std::vector<float> &C, int n) {
    hi.assign((size_t)n * (n / 2), 0);
    lo = hi;
    for (int p = 0; p < n; ++p)
      for (int i = 0; i < n / 2; ++i) {
        const size_t o = (size_t)p * (n / 2) + i;
        host_split(C[(size_t)fold_freq(p, n) * n + i], hi[o], lo[o]);
      }
  };
  // inverse: [3][n/2][n] from three [i][k] matrices (w: column scale or null)
  auto inv = [&](const std::vector<float> *M3[3], const std::vector<float> *w3[3], int n) {
    hi.assign((size_t)3 * (n / 2) * n, 0);
    lo = hi;
    for (int w = 0; w < 3; ++w)
      for (int i = 0; i < n / 2; ++i)
        for (int p = 0; p < n; ++p) {
          const int k = fold_freq(p, n);
          float v = (*M3[w])[(size_t)i * n + k];
          if (w3[w]) v = (float)((double)v * (double)(*w3[w])[k]);
          const size_t o = ((size_t)w * (n / 2) + i) * n + p;
          host_split(v, hi[o], lo[o]);
        }
  };
  int rc;
  fwd(Cn, ny);
  if ((rc = put(d.A1h, d.A1l))) return rc;
  fwd(Cm, nx);
  if ((rc = put(d.A2h, d.A2l))) return rc;
  const std::vector<float> *m3[3] = {&CTn, &STn, &CTn}, *w3[3] = {nullptr, &wv, nullptr};
  inv(m3, w3, ny);
  if ((rc = put(d.A3h, d.A3l))) return rc;
  const std::vector<float> *m4[3] = {&STm, &CTm, &CTm}, *w4[3] = {nullptr, nullptr, nullptr};
  inv(m4, w4, nx);
  if ((rc = put(d.A4h, d.A4l))) return rc;
  std::vector<float> t(std::max(nx, ny));
  auto perm = [&](float *dst, const std::vector<float> &src, int n) -> int {
    for (int p = 0; p < n; ++p) t[p] = src[fold_freq(p, n)];
    if (cudaMemcpy(dst, t.data(), sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(PLACE_ECUDA, "upload of the frequency tables failed");
    return PLACE_OK;
  };
  if ((rc = perm(d.wu_p, wu, nx)) || (rc = perm(d.cu_p, cu, nx)) || (rc = perm(d.wv_p, wv, ny)) ||
      (rc = perm(d.cv_p, cv, ny)))
    return rc;
  return PLACE_OK;
}

}  // namespace

extern "C" {

int place_create(const place_netlist *nl, const place_die *die, const place_bins *bins,
                 const place_params *params, void *stream, place_t **out) {
  NvtxRange nvtx_("place_create");
  if (out) *out = nullptr;
  if (!nl || !die || !bins || !out) return fail(PLACE_EINVAL, "null argument");
  place_params prm;
  if (params) prm = *params; else place_default_params(&prm);
  const int C = nl->n_cells, Mv = nl->n_movable, E = nl->n_nets, P = nl->n_pins;
  if (C <= 0 || Mv < 0 || Mv > C || E < 0 || P < 0)
    return fail(PLACE_EINVAL, "bad sizes: n_cells=%d n_movable=%d n_nets=%d n_pins=%d", C, Mv, E, P);
  if (C >= (1 << 30)) return fail(PLACE_EINVAL, "too many cells");
  if (!nl->w || !nl->h || !nl->x0 || !nl->y0 || !nl->net_ptr || (P > 0 && (!nl->pin_cell || !nl->pin_dx || !nl->pin_dy)))
    return fail(PLACE_EINVAL, "null netlist array");
  if (prm.n_copies < 1 || prm.n_copies > 4096) return fail(PLACE_EINVAL, "n_copies must be in [1, 4096]");
  if (prm.max_iters < 0) return fail(PLACE_EINVAL, "max_iters < 0");
  if (prm.max_backtracks < 0 || prm.max_backtracks > 64)
    return fail(PLACE_EINVAL, "max_backtracks must be in [0, 64]");
  if (prm.stretch != 0 && prm.stretch != 1) return fail(PLACE_EINVAL, "stretch must be 0 or 1");
  if (prm.autotune != 0 && prm.autotune != 1) return fail(PLACE_EINVAL, "autotune must be 0 or 1");
  if (prm.scatter_mode < -1 || prm.scatter_mode > 2)
    return fail(PLACE_EINVAL, "scatter_mode must be -1, 0, 1 or 2");
  if (prm.gemm_bn != 0 && prm.gemm_bn != 64 && prm.gemm_bn != 128)
    return fail(PLACE_EINVAL, "gemm_bn must be 0, 64 or 128");
  if (prm.wa_big_cap != 0 && (prm.wa_big_cap < 32 || prm.wa_big_cap > 6144))
    return fail(PLACE_EINVAL, "wa_big_cap must be 0 or in [32, 6144]");
  if (prm.gemm_split < 0 || prm.gemm_split > 2) return fail(PLACE_EINVAL, "gemm_split must be 0, 1 or 2");
  if (prm.wa_streams < 0 || prm.wa_streams > kMaxWaStreams)
    return fail(PLACE_EINVAL, "wa_streams must be 0, 1, 2 or 3");
  if (prm.dct_fold != 0 && prm.dct_fold != 1) return fail(PLACE_EINVAL, "dct_fold must be 0 or 1");
  if (prm.fillers != 0 && prm.fillers != 1) return fail(PLACE_EINVAL, "fillers must be 0 or 1");
  if (!(prm.macro_precond > 0.f) || !std::isfinite(prm.macro_precond))
    return fail(PLACE_EINVAL, "macro_precond must be positive and finite");
  prm.dct_mode = resolve_dct_mode(prm.dct_mode, bins->nx, bins->ny);
  if (prm.dct_mode != PLACE_DCT_FP32 && prm.dct_mode != PLACE_DCT_BF16X3)
    return fail(PLACE_EINVAL, "unknown dct_mode %d", prm.dct_mode);
  if (prm.dct_mode == PLACE_DCT_BF16X3 && (bins->nx % 128 || bins->ny % 128))
    return fail(PLACE_EINVAL, "the tensor-core spectral path needs bins in multiples of 128");
  const int nx = bins->nx, ny = bins->ny;
  if (nx < 16 || ny < 16 || nx % 16 || ny % 16 || nx > 8192 || ny > 8192)
    return fail(PLACE_EINVAL, "bins must be multiples of 16 in [16, 8192], got %dx%d", nx, ny);
  if (!(die->xh > die->xl) || !(die->yh > die->yl)) return fail(PLACE_EINVAL, "empty die");
  if (!(bins->target_density > 0.f)) return fail(PLACE_EINVAL, "target density must be > 0");

  // netlist checks
  if (nl->net_ptr[0] != 0 || nl->net_ptr[E] != P) return fail(PLACE_EINVAL, "net_ptr must start at 0 and end at n_pins");
  for (int e = 0; e < E; ++e)
    if (nl->net_ptr[e + 1] < nl->net_ptr[e]) return fail(PLACE_EINVAL, "net_ptr not monotone at net %d", e);
  for (int j = 0; j < P; ++j)
    if (nl->pin_cell[j] < 0 || nl->pin_cell[j] >= C) return fail(PLACE_EINVAL, "pin %d on cell %d out of range", j, nl->pin_cell[j]);
  double total_area = 0.0;
  for (int i = 0; i < C; ++i) {
    if (!(nl->w[i] > 0.f) || !(nl->h[i] > 0.f)) return fail(PLACE_EINVAL, "cell %d has non-positive size", i);
    if (!std::isfinite(nl->x0[i]) || !std::isfinite(nl->y0[i])) return fail(PLACE_EINVAL, "cell %d has a non-finite position", i);
    total_area += (double)nl->w[i] * (double)nl->h[i];
  }

  const int F = choose_frac_bits(die, total_area);
  if (F < 0) return fail(PLACE_ERANGE, "design does not fit the 64-bit fixed-point density range");
  const double s = std::ldexp(1.0, F);
  const double bw = (die->xh - die->xl) / nx, bh = (die->yh - die->yl) / ny;
  if (!is_integer(die->xl * s) || !is_integer(die->yl * s) || !is_integer(bw * s) || !is_integer(bh * s))
    return fail(PLACE_EINVAL, "die origin and bin size must be multiples of 2^-%d", F);

  place_t *h = new place_t();
  Dev &d = h->d;
  d.K = prm.n_copies;
  d.n_cells = C; d.n_mov = Mv; d.n_nets = E; d.n_pins = P;
  d.nx = nx; d.ny = ny; d.G = nx * ny;
  d.F = F;
  d.scale = (float)s;
  d.inv_scale = (float)std::ldexp(1.0, -F);
  d.inv_area_q = (float)std::ldexp(1.0, -2 * F);
  d.XL = (long long)(die->xl * s); d.YL = (long long)(die->yl * s);
  d.BW = (long long)(bw * s); d.BH = (long long)(bh * s);
  d.t = (double)bins->target_density;
  {
    // t = mant * 2^-shift exactly (24-bit mantissa of the float)
    int e = 0;
    double f = std::frexp((double)bins->target_density, &e);
    d.t_mant = (long long)std::ldexp(f, 24);
    d.t_shift = 24 - e;
    if (d.t_shift < 0 || d.t_shift > 60) {
      delete h;
      return fail(PLACE_EINVAL, "target density out of range");
    }
  }
  d.abin_q = (double)d.BW * (double)d.BH;
  {
    const unsigned __int128 tA = (unsigned __int128)(unsigned long long)d.t_mant *
                                 (unsigned __int128)(unsigned long long)(d.BW * d.BH);
    d.tA_lo = (unsigned long long)tA;
    d.tA_hi = (unsigned long long)(tA >> 64);
    const unsigned __int128 fl = tA >> d.t_shift;
    d.tA_floor = fl > (unsigned __int128)0x7fffffffffffffffull ? 0x7fffffffffffffffull
                                                                 : (unsigned long long)fl;
  }
  d.BW32 = (int)d.BW; d.BH32 = (int)d.BH;
  d.ibw_q = (float)(1.0 / (double)d.BW); d.ibh_q = (float)(1.0 / (double)d.BH);
  d.die_xl = die->xl; d.die_yl = die->yl; d.die_xh = die->xh; d.die_yh = die->yh;
  d.fxl = (float)die->xl; d.fyl = (float)die->yl; d.fxh = (float)die->xh; d.fyh = (float)die->yh;
  d.fbw = (float)bw; d.fbh = (float)bh; d.fibw = (float)(1.0 / bw); d.fibh = (float)(1.0 / bh);
  d.w_bin = std::sqrt(bw * bh);
  d.dref = (double)prm.hpwl_ref * (double)E * d.w_bin;
  d.prm = prm;
  d.has_net_w = nl->net_w ? 1 : 0;
  d.tc = prm.dct_mode == PLACE_DCT_BF16X3 ? 1 : 0;
  d.bfly = use_fold(d.tc, prm.dct_fold, bins->nx, bins->ny);
  h->stream = (cudaStream_t)stream;

  // quantised sizes and movable area
  std::vector<int> Wq(C), Hq(C);
  unsigned __int128 mov_area_q = 0;  // exact; converted to double once
  for (int i = 0; i < C; ++i) {
    double wq = std::nearbyint((double)nl->w[i] * s), hq = std::nearbyint((double)nl->h[i] * s);
    if (wq < 1 || hq < 1 || wq >= 2147483647.0 || hq >= 2147483647.0) {
      delete h;
      return fail(PLACE_ERANGE, "cell %d size out of the fixed-point range", i);
    }
    Wq[i] = (int)wq; Hq[i] = (int)hq;
    if (i < Mv) mov_area_q += (unsigned __int128)((unsigned long long)Wq[i] * (unsigned long long)Hq[i]);
  }
  d.mov_area_q = mov_area_q > 0 ? (double)mov_area_q : 1.0;

  // filler cells; the library's cell order is [movable | fillers | fixed]
  FillPlan fp;
  if (prm.fillers) fp = plan_fillers(nl, die, bins, F, mov_area_q);
  if ((long long)C + fp.n >= (1LL << 30)) {
    delete h;
    return fail(PLACE_ERANGE, "too many filler cells (%lld)", fp.n);
  }
  const int nf = (int)fp.n;
  const int Ci = C + nf, Mo = Mv + nf;  // library cells, optimiser cells
  auto ci = [&](int i) { return i < Mv ? i : i + nf; };  // design cell -> library cell
  d.n_cells = Ci; d.n_mov = Mo; d.n_real = Mv; d.n_fill = nf;
  d.Gm = nf ? 2 * d.G : d.G;
  d.fill_area_q = (double)nf * (double)fp.Wf * (double)fp.Hf;
  std::vector<float> wi(Ci), hi(Ci);
  std::vector<int> Wqi(Ci), Hqi(Ci);
  std::vector<unsigned char> macro(Ci, 0);
  std::vector<float2> xy0(Ci);
  for (int i = 0; i < C; ++i) {
    const int k = ci(i);
    wi[k] = nl->w[i]; hi[k] = nl->h[i];
    Wqi[k] = Wq[i]; Hqi[k] = Hq[i];
    xy0[k] = make_float2(nl->x0[i], nl->y0[i]);
    if (nl->is_macro) macro[k] = nl->is_macro[i] ? 1 : 0;
  }
  {
    const double wf = fp.Wf * std::ldexp(1.0, -F), hf = fp.Hf * std::ldexp(1.0, -F);
    filler_start(nf, die, wf, hf, xy0.data() + Mv);
    for (int j = 0; j < nf; ++j) {
      wi[Mv + j] = (float)wf; hi[Mv + j] = (float)hf;
      Wqi[Mv + j] = fp.Wf; Hqi[Mv + j] = fp.Hf;
    }
  }

  // nets grouped by degree class (stable), pins in the new net order
  std::vector<int> order(E);
  {
    std::vector<int> cnt(6, 0);
    for (int e = 0; e < E; ++e) cnt[degree_class(nl->net_ptr[e + 1] - nl->net_ptr[e]) + 1]++;
    for (int c = 0; c < 5; ++c) cnt[c + 1] += cnt[c];
    d.n_cls = 5;
    for (int c = 0; c <= 5; ++c) d.cls_begin[c] = cnt[c];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int e = 0; e < E; ++e) order[pos[degree_class(nl->net_ptr[e + 1] - nl->net_ptr[e])]++] = e;
    // nets above 256 pins (one block each) by descending degree: the longest
    // start first, which balances the blocks
    auto deg = [&](int e) { return nl->net_ptr[e + 1] - nl->net_ptr[e]; };
    std::stable_sort(order.begin() + d.cls_begin[4], order.begin() + d.cls_begin[5],
                     [&](int a, int b) { return deg(a) > deg(b); });
    // the other classes by their lowest cell index, whose pin goes first
    // (below): the first pins of the nets a warp handles then lie on nearby
    // cells, so their position gathers and gradient reductions share sectors
    std::vector<int> min_cell(E, 0);
    for (int e = 0; e < E; ++e) {
      int m = C;
      for (int j = nl->net_ptr[e]; j < nl->net_ptr[e + 1]; ++j) m = std::min(m, nl->pin_cell[j]);
      min_cell[e] = m;
    }
    // the one-thread class by degree first, so that a warp's nets take one
    // path (2-pin nets a closed form) and only the warps at the boundaries
    // mix them
    std::stable_sort(order.begin() + d.cls_begin[0], order.begin() + d.cls_begin[1],
                     [&](int a, int b) {
                       return deg(a) != deg(b) ? deg(a) < deg(b) : min_cell[a] < min_cell[b];
                     });
    // the group classes in two sub-ranges, each by lowest cell: the nets of
    // up to half the class's lane slots first (they run on half the lanes)
    for (int c = 1; c < 4; ++c) {
      const int half = kGroupHalfDeg[c];
      std::stable_sort(order.begin() + d.cls_begin[c], order.begin() + d.cls_begin[c + 1],
                       [&](int a, int b) {
                         const bool ha = deg(a) > half, hb = deg(b) > half;
                         return ha != hb ? hb : min_cell[a] < min_cell[b];
                       });
    }
    for (int c = 0; c < 8; ++c) d.cls_split[c] = c < 6 ? d.cls_begin[std::min(c + 1, 5)] : 0;
    for (int c = 1; c < 4; ++c) {
      int e = d.cls_begin[c];
      while (e < d.cls_begin[c + 1] && deg(order[e]) <= kGroupHalfDeg[c]) ++e;
      d.cls_split[c] = e;
    }
  }
  std::vector<int> net_ptr(E + 1), pin_cell(P);
  std::vector<float2> pin_off(P);
  std::vector<float> net_w;
  if (nl->net_w) net_w.resize(E);
  net_ptr[0] = 0;
  for (int ne = 0; ne < E; ++ne) {
    int e = order[ne];
    int p0 = nl->net_ptr[e], p1 = nl->net_ptr[e + 1];
    int q = net_ptr[ne];
    int jmin = p0;  // the pin on the lowest cell index goes first
    for (int j = p0 + 1; j < p1; ++j)
      if (nl->pin_cell[j] < nl->pin_cell[jmin]) jmin = j;
    for (int j = p0; j < p1; ++j, ++q) {
      const int src = j == p0 ? jmin : (j == jmin ? p0 : j);
      pin_cell[q] = ci(nl->pin_cell[src]);
      pin_off[q] = make_float2(nl->pin_dx[src], nl->pin_dy[src]);
    }
    net_ptr[ne + 1] = q;
    if (nl->net_w) net_w[ne] = nl->net_w[e];
  }
  // pins per movable cell, and the fixed-point scale 2^Fg of the packed WA
  // gradient sums.  One pin's gradient on a net of n pins is the difference
  // of two softmax-weighted terms w_j (1 - t_j + r), with t_j >= 0 and
  // r = sum w t = H(w) - ln S <= ln n (S >= 1, entropy H <= ln n), so
  // |gradient| <= 2 (1 + 1/e + ln n) < 3 + 2 ln n per unit net weight.
  // Fg keeps every cell's sum of those bounds below 0.9 * 2^31.
  std::vector<int> cell_npins(std::max(Mv, 1), 0);
  std::vector<double> gbound(std::max(Mv, 1), 0.0);
  for (int e = 0; e < E; ++e) {
    const int deg = net_ptr[e + 1] - net_ptr[e];
    const double b = (3.0 + 2.0 * std::log((double)std::max(deg, 1))) *
                     (nl->net_w ? std::fabs((double)net_w[e]) : 1.0);
    for (int j = net_ptr[e]; j < net_ptr[e + 1]; ++j)
      if (pin_cell[j] < Mv) {
        cell_npins[pin_cell[j]]++;
        gbound[pin_cell[j]] += b;
      }
  }
  double gmax = 0.0;
  for (int i = 0; i < Mv; ++i) gmax = std::max(gmax, gbound[i]);
  int Fg = 24;
  while (Fg > 0 && gmax * std::ldexp(1.0, Fg) >= 0.9 * 2147483648.0) --Fg;
  if (Fg < 10) {
    delete h;
    return fail(PLACE_ERANGE, "a movable cell carries too many pins (gradient bound %.3g) for "
                "the 32-bit fixed-point wirelength-gradient sums", gmax);
  }
  d.gq = (float)std::ldexp(1.0, Fg);
  d.giq = (float)std::ldexp(1.0, -Fg);
  int max_deg = 0;
  for (int e = 0; e < E; ++e) max_deg = std::max(max_deg, net_ptr[e + 1] - net_ptr[e]);
  d.wa_big_cap = prm.wa_big_cap ? prm.wa_big_cap : std::min(std::max(max_deg, 1), kBigCapMax);
  d.wa_streams = prm.wa_streams ? prm.wa_streams : 1;  // fixed rule: one chain
  d.scat_t1 = kScatterMergedBelow;
  d.scat_t2 = kScatterTableBelow;
  d.scat_force = prm.scatter_mode;
  // pins and charge per optimiser cell for the preconditioner
  // max(1, pins_i + lambda area_i); a movable macro's charge is weighted by
  // macro_precond
  std::vector<float> npins(std::max(Mo, 1), 0.f), area(std::max(Mo, 1));
  for (int i = 0; i < Mo; ++i) {
    if (i < Mv) npins[i] = (float)cell_npins[i];
    area[i] = (float)((double)wi[i] * (double)hi[i] * (i < Mv && macro[i] ? (double)prm.macro_precond : 1.0));
  }
  h->n_cand_all = Mv;
  h->n_cand_macro = 0;
  for (int i = 0; i < Mv; ++i) h->n_cand_macro += macro[i];
  if (h->n_cand_macro > 0) {
    // WireMask tables: the movable macros by decreasing area (exact in
    // double; ties keep index order), each macro's nets as library indices
    // in netlist order, and the obstacle list (fixed cells, then the macros)
    std::vector<int> lib_of(E);
    for (int ne = 0; ne < E; ++ne) lib_of[order[ne]] = ne;
    std::vector<int> &mo = h->wm_order;
    for (int i = 0; i < Mv; ++i)
      if (macro[i]) mo.push_back(i);
    std::stable_sort(mo.begin(), mo.end(), [&](int a, int b) {
      return (double)nl->w[a] * (double)nl->h[a] > (double)nl->w[b] * (double)nl->h[b];
    });
    std::vector<int> slot(C, -1);
    for (size_t t = 0; t < mo.size(); ++t) slot[mo[t]] = (int)t;
    std::vector<std::vector<int>> nets(mo.size());
    for (int e = 0; e < E; ++e)
      for (int j = nl->net_ptr[e]; j < nl->net_ptr[e + 1]; ++j) {
        const int t = slot[nl->pin_cell[j]];
        if (t >= 0 && (nets[t].empty() || nets[t].back() != lib_of[e])) nets[t].push_back(lib_of[e]);
      }
    h->wm_ptr.assign(1, 0);
    for (size_t t = 0; t < mo.size(); ++t) {
      h->wm_net.insert(h->wm_net.end(), nets[t].begin(), nets[t].end());
      h->wm_ptr.push_back((int)h->wm_net.size());
      h->wm_max_nets = std::max(h->wm_max_nets, (int)nets[t].size());
    }
    for (int i = Mv; i < C; ++i) h->wm_obst.push_back(ci(i));
    h->wm_obst.insert(h->wm_obst.end(), mo.begin(), mo.end());
  }

  // launch plan
  d.cell_blocks = std::max(1, std::min((Mo + kThreads - 1) / kThreads, kMaxCellBlocks));
  d.wa_blocks_total = 0;
  for (int c = 0; c < 5; ++c) {
    int n = d.cls_begin[c + 1] - d.cls_begin[c];
    int nb = c < 4 ? (n + kNetsPerBlock[c] - 1) / kNetsPerBlock[c] : n;
    nb = std::min(nb, c < 4 ? kMaxCellBlocks : kMaxBigNetBlocks);
    d.wa_blocks[c] = nb;
    d.wa_block_base[c] = d.wa_blocks_total;
    d.wa_blocks_total += nb;
  }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || d.sms <= 0)
      d.sms = 152;
    // the cell-gradient kernel runs as one resident wave (grid-stride)
    d.cg_blocks = std::max(1, std::min(d.cell_blocks, d.sms * cell_grad_blocks_per_sm()));
  }
  // four blocks per SM: more bins per thread amortise the per-block exact
  // reductions of the density finish (measured on the 2.1M-cell design:
  // 0.0816 -> 0.0783 ms for the density stage at iteration 5 against 1216
  // blocks; 304 blocks were in between)
  d.bin_blocks = std::max(1, std::min((d.G + kThreads - 1) / kThreads, 4 * std::max(d.sms, 1)));
  d.nb_red = std::max(std::max(2 * d.cell_blocks + 2, d.bin_blocks), std::max(d.wa_blocks_total, 1));
  int sn = 2;
  while (sn < Ci) sn <<= 1;
  d.sort_n = sn;

  // device memory: one allocation carved into arrays
  Arena a;
  layout(d, a, d.K);
  h->mem_bytes = a.off + 256;
  // stream-ordered allocation: creating and destroying handles (as the
  // job server does while other jobs run) never synchronises the device
  cudaError_t e = cudaMallocAsync(&h->mem, h->mem_bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // usable by the uploads below
  if (e != cudaSuccess) {
    delete h;
    return fail(PLACE_ENOMEM, "device allocation of %zu bytes failed: %s", (size_t)a.off, cudaGetErrorString(e));
  }
  a = Arena();
  a.base = (char *)h->mem;
  layout(d, a, d.K);

  int rc = PLACE_OK;
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (rc != PLACE_OK || bytes == 0) return;
    cudaError_t ce = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) rc = fail(PLACE_ECUDA, "upload failed: %s", cudaGetErrorString(ce));
  };
  up(d.net_ptr, net_ptr.data(), sizeof(int) * (E + 1));
  up(d.pin_cell, pin_cell.data(), sizeof(int) * P);
  up(d.pin_off, pin_off.data(), sizeof(float2) * P);
  up(d.w, wi.data(), sizeof(float) * Ci);
  up(d.h, hi.data(), sizeof(float) * Ci);
  up(d.Wq, Wqi.data(), sizeof(int) * Ci);
  up(d.Hq, Hqi.data(), sizeof(int) * Ci);
  {
    std::vector<float2> whv(std::max(Ci, 1)), pav(std::max(Mo, 1));
    for (int i = 0; i < Ci; ++i) whv[i] = make_float2(wi[i], hi[i]);
    for (int i = 0; i < Mo; ++i) pav[i] = make_float2(npins[i], area[i]);
    up(d.wh, whv.data(), sizeof(float2) * Ci);
    up(d.pa, pav.data(), sizeof(float2) * Mo);
  }
  up(d.is_macro, macro.data(), Ci);
  if (d.st) {
    // density stretching: along each axis a cell narrower than sqrt(2) bins
    // widens to rint(sqrt(2) BW) about its centre (shift floor((W' - W) / 2));
    // its density scale is R = floor(W H 2^31 / (W' H'))
    const long long ws = (long long)std::nearbyint(std::sqrt(2.0) * (double)d.BW);
    const long long hs = (long long)std::nearbyint(std::sqrt(2.0) * (double)d.BH);
    std::vector<int4> st(std::max(Mo, 1));
    std::vector<unsigned int> sR(std::max(Mo, 1));
    for (int i = 0; i < Mo; ++i) {
      const long long W2 = std::max<long long>(Wqi[i], ws), H2 = std::max<long long>(Hqi[i], hs);
      st[i] = make_int4((int)((W2 - Wqi[i]) >> 1), (int)((H2 - Hqi[i]) >> 1), (int)W2, (int)H2);
      const unsigned __int128 num = ((unsigned __int128)((unsigned long long)Wqi[i] * (unsigned long long)Hqi[i])) << 31;
      sR[i] = (unsigned int)(num / (unsigned __int128)((unsigned long long)W2 * (unsigned long long)H2));
    }
    up(d.st, st.data(), sizeof(int4) * Mo);
    up(d.sR, sR.data(), sizeof(unsigned int) * Mo);
  }
  if (d.net_w) up(d.net_w, net_w.data(), sizeof(float) * E);
  {
    std::vector<float> Cn, CTn, Sn, STn, Cm, CTm, Sm, STm, wu, wv, cu, cv;
    host_dct_tables(ny, bh, Cn, CTn, Sn, STn, wv, cv);
    host_dct_tables(nx, bw, Cm, CTm, Sm, STm, wu, cu);
    up(d.Cn, Cn.data(), sizeof(float) * Cn.size());
    up(d.CTn, CTn.data(), sizeof(float) * CTn.size());
    // G3 for Ey uses S_N[y][v] = sin(pi v (y+1/2)/N): the "ST" layout [i][k]
    up(d.STn, STn.data(), sizeof(float) * STn.size());
    up(d.Cm, Cm.data(), sizeof(float) * Cm.size());
    up(d.CTm, CTm.data(), sizeof(float) * CTm.size());
    up(d.STm, STm.data(), sizeof(float) * STm.size());
    up(d.wu, wu.data(), sizeof(float) * nx);
    up(d.wv, wv.data(), sizeof(float) * ny);
    up(d.cu, cu.data(), sizeof(float) * nx);
    up(d.cv, cv.data(), sizeof(float) * ny);
    if (rc == PLACE_OK && d.bfly)
      rc = upload_fold_tables(d, h->stream, Cn, CTn, STn, Cm, CTm, STm, wu, wv, cu, cv);
  }
  for (int c = 0; c < d.K && rc == PLACE_OK; ++c) up(d.xy + (size_t)c * Ci, xy0.data(), sizeof(float2) * Ci);
  if (rc != PLACE_OK) {
    place_destroy(h);
    return rc;
  }
  cudaError_t ce = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&h->cap3, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&h->cap4, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_join3, cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    place_destroy(h);
    return fail(PLACE_ECUDA, "stream create: %s", cudaGetErrorString(ce));
  }
  ce = cudaMemsetAsync(d.E, 0, sizeof(float) * (size_t)d.K * 3 * d.G, h->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d.Fmap, 0, sizeof(long long) * d.G, h->stream);
  if (ce == cudaSuccess)
    ce = cudaMemsetAsync(d.gacc, 0, sizeof(unsigned long long) * (size_t)d.K * std::max(Mo, 1), h->stream);
  if (ce == cudaSuccess && wa_prepare(d.wa_big_cap)) ce = cudaErrorInvalidValue;
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d.cs, 0, sizeof(CopyState) * d.K, h->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d.ctr, 0, sizeof(unsigned int) * d.K * C_COUNT, h->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d.err, 0, 4 * sizeof(int), h->stream);
  if (ce != cudaSuccess) {
    place_destroy(h);
    return fail(PLACE_ECUDA, "memset: %s", cudaGetErrorString(ce));
  }
  if (d.tc && (rc = setup_tc(h)) != PLACE_OK) {
    place_destroy(h);
    return rc;
  }
  launch_scatter_fixed(d, d.xy, Mo, Ci, reinterpret_cast<unsigned long long *>(d.Fmap), h->stream);
  rc = enqueue_reset(h, 0, d.K);
  if (rc == PLACE_OK) {
    ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) rc = fail(PLACE_ECUDA, "create: %s", cudaGetErrorString(ce));
  }
  if (rc == PLACE_OK && prm.autotune) {
    // time the candidates on this design, then put copy 0 and every
    // optimiser back to the start
    NvtxRange nvtx_tune("autotune");
    TuneOut to{};
    TuneCtx tctx{h, xy0.data()};
    const TuneHooks hooks{encode_tc_maps_cb, time_iters_cb, &tctx};
    int trc = autotune(d, max_deg, h->stream, hooks, &to);
    drop_graph(h);  // captured for a candidate; the first step captures the final choice
    if (trc) {
      rc = fail(trc, "autotuning failed: %s", cudaGetErrorString(cudaGetLastError()));
    } else {
      h->autotuned = 1;
      h->autotune_ms = to.ms;
      for (int c = 0; c < d.K && rc == PLACE_OK; ++c) up(d.xy + (size_t)c * Ci, xy0.data(), sizeof(float2) * Ci);
      if (rc == PLACE_OK) rc = enqueue_reset(h, 0, d.K);
      if (rc == PLACE_OK) {
        ce = cudaStreamSynchronize(h->stream);
        if (ce != cudaSuccess) rc = fail(PLACE_ECUDA, "create: %s", cudaGetErrorString(ce));
      }
    }
  }
  if (rc != PLACE_OK) {
    place_destroy(h);
    return rc;
  }
  *out = h;
  return PLACE_OK;
}

int place_get_info(const place_t *h, place_info *o) {
  if (!h || !o) return fail(PLACE_EINVAL, "null argument");
  const Dev &d = h->d;
  o->n_cells = d.n_cells - d.n_fill; o->n_movable = d.n_real; o->n_nets = d.n_nets; o->n_pins = d.n_pins;
  o->n_fillers = d.n_fill;
#ifdef PLACE_DEBUG_BOUNDS
  o->bounds_checked = 1;
#else
  o->bounds_checked = 0;
#endif
  o->nx = d.nx; o->ny = d.ny; o->n_copies = d.K;
  o->frac_bits = d.F;
  o->bin_w_q = d.BW; o->bin_h_q = d.BH;
  o->bin_w = (d.die_xh - d.die_xl) / d.nx;
  o->bin_h = (d.die_yh - d.die_yl) / d.ny;
  o->device_bytes = (int64_t)h->mem_bytes;
  int wa = 0;
  for (int c = 0; c < d.n_cls; ++c) wa += d.wa_blocks[c] > 0;
  // scatter, finish, 4 GEMMs, WA classes, cell grad, precond0, update; the
  // stretched scatter with density stretching, the step redo with backtracking
  // the steady graph (the first iteration after a reset adds k_precond0)
  o->kernels_per_iter = 2 + 4 + wa + 2 + (d.Ms ? 1 : 0) + (d.up ? 1 : 0);
  o->dct_mode = d.tc ? PLACE_DCT_BF16X3 : PLACE_DCT_FP32;
  for (int s = 0; s < 4; ++s) {
    o->gemm_bn[s] = d.tc ? d.tc_bn[s] : 0;
    o->gemm_split[s] = d.tc ? d.tc_split[s] : 0;
  }
  o->wa_big_cap = d.wa_big_cap;
  o->autotuned = h->autotuned;
  o->scatter_t1 = d.scat_t1;
  o->scatter_t2 = d.scat_t2;
  o->autotune_ms = h->autotune_ms;
  o->wa_streams = d.wa_streams;
  o->dct_fold = d.bfly;
  return PLACE_OK;
}

int place_step(place_t *h, int32_t n_iters, int32_t *converged) {
  NvtxRange nvtx_("place_step");
  if (!h) return fail(PLACE_EINVAL, "null handle");
  if (n_iters < 0) return fail(PLACE_EINVAL, "n_iters < 0");
  if (n_iters > 0) {
    int rc = ensure_graph(h);
    if (rc) return rc;
    for (int i = 0; i < n_iters; ++i) CK(launch_iter(h));
  }
  if (converged) {
    std::vector<CopyState> cs(h->d.K);
    CK(cudaMemcpyAsync(cs.data(), h->d.cs, sizeof(CopyState) * h->d.K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < h->d.K; ++c) converged[c] = cs[c].stopped;
    return check_dev_err(h);
  }
  return PLACE_OK;
}

int place_step_multi(place_t *const *hs, int32_t n, int32_t n_iters, int32_t *converged) {
  NvtxRange nvtx_("place_step_multi");
  if (!hs || n < 1) return fail(PLACE_EINVAL, "need at least one handle");
  if (n_iters < 0) return fail(PLACE_EINVAL, "n_iters < 0");
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return fail(PLACE_EINVAL, "null handle %d", i);
  if (n_iters > 0) {
    for (int i = 0; i < n; ++i) {
      int rc = ensure_graph(hs[i]);
      if (rc) return rc;
    }
    for (int it = 0; it < n_iters; ++it)
      for (int i = 0; i < n; ++i) CK(launch_iter(hs[i]));
  }
  if (converged) {
    int off = 0;
    for (int i = 0; i < n; ++i) {
      int rc = place_step(hs[i], 0, converged + off);
      if (rc) return rc;
      off += hs[i]->d.K;
    }
  }
  return PLACE_OK;
}

int place_step_timed(place_t *h, int32_t n_iters, float *stage_ms) {
  NvtxRange nvtx_("place_step_timed");
  if (!h || !stage_ms) return fail(PLACE_EINVAL, "null argument");
  const Dev &d = h->d;
  const int K = d.K;
  cudaStream_t st = h->stream;
  cudaEvent_t ev[PLACE_N_STAGES + 1];
  for (auto &e : ev) CK(cudaEventCreate(&e));
  std::vector<double> acc(PLACE_N_STAGES, 0.0);
  int rc = PLACE_OK;
  for (int it = 0; it < n_iters && rc == PLACE_OK; ++it) {
    cudaEventRecord(ev[0], st);
    cudaMemsetAsync(d.M, 0, sizeof(unsigned long long) * (size_t)d.Gm * K, st);
    launch_scatter(d, 0, K, 0, st);
    launch_density_finish(d, 0, K, FIN_ITER, st);
    cudaEventRecord(ev[1], st);
    launch_spectral(d, 0, K, 0, 0, st);
    cudaEventRecord(ev[2], st);
    launch_wa(d, 0, K, 0, nullptr, st);
    cudaEventRecord(ev[3], st);
    launch_cell_grad(d, 0, K, 0, st);
    cudaEventRecord(ev[4], st);
    launch_precond0(d, 0, K, st);
    launch_update(d, 0, K, st);
    cudaEventRecord(ev[5], st);
    cudaError_t e = cudaEventSynchronize(ev[5]);
    if (e != cudaSuccess) { rc = fail(PLACE_ECUDA, "timed step: %s", cudaGetErrorString(e)); break; }
    for (int s = 0; s < PLACE_N_STAGES; ++s) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
      acc[s] += ms;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  CKL();
  if ((rc = check_dev_err(h))) return rc;
  for (int s = 0; s < PLACE_N_STAGES; ++s) stage_ms[s] += (float)acc[s];
  return PLACE_OK;
}

int place_test_wait_timeout(place_t *h) {
  if (!h) return fail(PLACE_EINVAL, "null handle");
  if (!h->d.tc) return fail(PLACE_EINVAL, "the handle has no tensor-core spectral path");
  NvtxRange nvtx_("place_test_wait_timeout");
  launch_spectral_tc_stalled(h->d, h->stream);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  const int rc = check_dev_err(h);
  // the kernel ended on its own: clear the flag, the handle stays usable
  CK(cudaMemsetAsync(h->d.err, 0, sizeof(int), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

int place_measure_scatter_floor(place_t *h, int32_t reps, float *ms_scatter, float *ms_floor) {
  if (!h || !ms_scatter || !ms_floor) return fail(PLACE_EINVAL, "null argument");
  if (reps < 1) return fail(PLACE_EINVAL, "reps < 1");
  NvtxRange nvtx_("place_measure_scatter_floor");
  const Dev &d = h->d;
  cudaStream_t st = h->stream;
  const size_t mbytes = sizeof(unsigned long long) * (size_t)d.Gm * d.K;
  cudaEvent_t ev[4];
  for (auto &e : ev) CK(cudaEventCreate(&e));
  // the scatter as the iteration runs it (the way its copies' last pass
  // chose), then the floor kernel, each after a cleared map
  cudaMemsetAsync(d.M, 0, mbytes, st);
  launch_scatter_main(d, 0, d.K, 1, st);  // warm-up
  cudaMemsetAsync(d.M, 0, mbytes, st);
  launch_scatter_floor(d, 0, d.K, st);
  float t[2] = {0.f, 0.f};
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaMemsetAsync(d.M, 0, mbytes, st);
    cudaEventRecord(ev[0], st);
    launch_scatter_main(d, 0, d.K, 1, st);
    cudaEventRecord(ev[1], st);
    cudaMemsetAsync(d.M, 0, mbytes, st);
    cudaEventRecord(ev[2], st);
    launch_scatter_floor(d, 0, d.K, st);
    cudaEventRecord(ev[3], st);
    e = cudaEventSynchronize(ev[3]);
    float a = 0.f, b = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[2], ev[3]);
    t[0] += a;
    t[1] += b;
  }
  // the map is scratch here: the next density pass clears and rebuilds it
  cudaMemsetAsync(d.M, 0, mbytes, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (auto &x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return fail(PLACE_ECUDA, "scatter floor: %s", cudaGetErrorString(e));
  CKL();
  *ms_scatter = t[0] / reps;
  *ms_floor = t[1] / reps;
  return check_dev_err(h);
}

int place_test_bounds_check(place_t *h) {
  if (!h) return fail(PLACE_EINVAL, "null handle");
#ifndef PLACE_DEBUG_BOUNDS
  return fail(PLACE_EINVAL, "this library was built without index checks");
#else
  NvtxRange nvtx_("place_test_bounds_check");
  launch_test_bounds(h->d, h->stream);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return check_dev_err(h);  // reports and clears the failed check
#endif
}

int place_measure_wa_floor(place_t *h, int32_t reps, float *ms) {
  if (!h || !ms) return fail(PLACE_EINVAL, "null argument");
  if (reps < 1) return fail(PLACE_EINVAL, "reps < 1");
  const Dev &d = h->d;
  cudaStream_t st = h->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  launch_wa_floor(d, 0, d.K, st);  // warm-up
  cudaEventRecord(e0, st);
  for (int i = 0; i < reps; ++i) launch_wa_floor(d, 0, d.K, st);
  cudaEventRecord(e1, st);
  // the floor kernel added into the gradient sums: clear them for the next pass
  cudaMemsetAsync(d.gacc, 0, sizeof(unsigned long long) * (size_t)d.K * std::max(d.n_mov, 1), st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(PLACE_ECUDA, "floor measurement: %s", cudaGetErrorString(e));
  CKL();
  *ms = t / reps;
  return PLACE_OK;
}

int place_get_state(place_t *h, int32_t copy, place_state *o) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (!o) return fail(PLACE_EINVAL, "null output");
  CopyState cs;
  CK(cudaMemcpyAsync(&cs, h->d.cs + copy, sizeof cs, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if ((rc = check_dev_err(h))) return rc;
  o->iter = cs.k; o->converged = cs.converged; o->stopped = cs.stopped;
  o->backtracks = cs.n_back_total;
  o->lambda = cs.lam; o->gamma = cs.gamma; o->alpha = cs.alpha; o->a = cs.a;
  o->overflow = cs.tau; o->hpwl_wa = cs.hpwl; o->bins_effective = cs.n_eff;
  return PLACE_OK;
}

int place_get_history(place_t *h, int32_t copy, place_iter_record *out, int32_t cap, int32_t *n) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (cap < 0) return fail(PLACE_EINVAL, "cap < 0");
  const Dev &d = h->d;
  CopyState cs;
  CK(cudaMemcpyAsync(&cs, d.cs + copy, sizeof cs, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int kept = std::min(cs.n_hist, d.hist_cap);
  if (n) *n = kept;
  const int m = std::min(kept, (int)cap);
  if (out && m > 0) {
    // the last m records, oldest first: ring slots (n_hist - m .. n_hist - 1) mod cap
    std::vector<place_iter_record> ring(d.hist_cap);
    CK(cudaMemcpy(ring.data(), d.hist + (size_t)copy * d.hist_cap,
                  sizeof(place_iter_record) * d.hist_cap, cudaMemcpyDeviceToHost));
    for (int i = 0; i < m; ++i) out[i] = ring[(cs.n_hist - m + i) % d.hist_cap];
  }
  return PLACE_OK;
}

}  // extern "C"

namespace {

// Checkpoint layout: a header, the copy's CopyState, then its arrays in the
// order of ckpt_arrays (each padded to 8 bytes), then the history ring.
struct CkptHeader {
  char magic[8];                 // "HYBROCK1"
  int32_t version;               // 3: (x, y) pairs interleaved; the step-norm partials
  int32_t n_cells, n_mov, n_real, n_fill, n_nets, n_pins, nx, ny, frac_bits, hist_cap;
  int32_t norm_blocks;           // step-norm partials saved (blocks of the update kernel)
  int32_t has_up;                // backtracking arrays present
  int32_t state_bytes;           // sizeof(CopyState)
  double dref, w_bin;            // the schedule's reference step and bin size
};

struct CkptArray {
  void *dev;
  size_t bytes;
};

std::vector<CkptArray> ckpt_arrays(const Dev &d, int c) {
  const size_t C = d.n_cells, Mo = d.n_mov;
  std::vector<CkptArray> v = {
      {d.xy + c * C, sizeof(float2) * C},
      {d.u + c * Mo, sizeof(float2) * Mo},
      {d.g[0] + c * Mo, sizeof(float2) * Mo}, {d.g[1] + c * Mo, sizeof(float2) * Mo},
      // the last step's |v_k - v_{k-1}|^2 partials (one per update block)
      {d.part + ((size_t)c * S_COUNT + S_DV2) * d.nb_red, sizeof(double) * d.cell_blocks},
      {d.gwx + c * Mo, sizeof(float) * Mo}, {d.gwy + c * Mo, sizeof(float) * Mo},
      {d.gdx + c * Mo, sizeof(float) * Mo}, {d.gdy + c * Mo, sizeof(float) * Mo},
      {d.gacc + c * Mo, sizeof(unsigned long long) * Mo},
      {d.hist + (size_t)c * d.hist_cap, sizeof(place_iter_record) * d.hist_cap}};
  if (d.up) {
    v.push_back({d.vp + c * Mo, sizeof(float2) * Mo});
    v.push_back({d.up + c * Mo, sizeof(float2) * Mo});
  }
  return v;
}

size_t pad8(size_t n) { return (n + 7) & ~size_t(7); }

CkptHeader ckpt_header(const Dev &d) {
  CkptHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, "HYBROCK1", 8);
  hd.version = 3;
  hd.norm_blocks = d.cell_blocks;
  hd.n_cells = d.n_cells; hd.n_mov = d.n_mov; hd.n_real = d.n_real; hd.n_fill = d.n_fill;
  hd.n_nets = d.n_nets; hd.n_pins = d.n_pins; hd.nx = d.nx; hd.ny = d.ny;
  hd.frac_bits = d.F; hd.hist_cap = d.hist_cap;
  hd.has_up = d.up ? 1 : 0;
  hd.state_bytes = (int32_t)sizeof(CopyState);
  hd.dref = d.dref; hd.w_bin = d.w_bin;
  return hd;
}

size_t ckpt_bytes(const Dev &d) {
  size_t n = pad8(sizeof(CkptHeader)) + pad8(sizeof(CopyState));
  for (const CkptArray &a : ckpt_arrays(d, 0)) n += pad8(a.bytes);
  return n;
}

}  // namespace

extern "C" {

int place_checkpoint_bytes(const place_t *h, int64_t *bytes) {
  if (!h) return fail(PLACE_EINVAL, "null handle");
  if (!bytes) return fail(PLACE_EINVAL, "null output");
  *bytes = (int64_t)ckpt_bytes(h->d);
  return PLACE_OK;
}

int place_checkpoint_save(place_t *h, int32_t copy, void *buf, int64_t cap) {
  NvtxRange nvtx_("place_checkpoint_save");
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  const Dev &d = h->d;
  if (!buf) return fail(PLACE_EINVAL, "null buffer");
  if (cap < (int64_t)ckpt_bytes(d))
    return fail(PLACE_EINVAL, "buffer of %lld bytes, the checkpoint needs %lld", (long long)cap,
                (long long)ckpt_bytes(d));
  unsigned char *p = static_cast<unsigned char *>(buf);
  const CkptHeader hd = ckpt_header(d);
  std::memcpy(p, &hd, sizeof hd);
  p += pad8(sizeof hd);
  CK(cudaMemcpyAsync(p, d.cs + copy, sizeof(CopyState), cudaMemcpyDeviceToHost, h->stream));
  p += pad8(sizeof(CopyState));
  for (const CkptArray &a : ckpt_arrays(d, copy)) {
    CK(cudaMemcpyAsync(p, a.dev, a.bytes, cudaMemcpyDeviceToHost, h->stream));
    p += pad8(a.bytes);
  }
  CK(cudaStreamSynchronize(h->stream));
  return check_dev_err(h);
}

int place_checkpoint_load(place_t *h, int32_t copy, const void *buf, int64_t bytes) {
  NvtxRange nvtx_("place_checkpoint_load");
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  const Dev &d = h->d;
  if (!buf) return fail(PLACE_EINVAL, "null buffer");
  if (bytes < (int64_t)ckpt_bytes(d))
    return fail(PLACE_EINVAL, "checkpoint of %lld bytes, this handle's needs %lld",
                (long long)bytes, (long long)ckpt_bytes(d));
  const unsigned char *p = static_cast<const unsigned char *>(buf);
  CkptHeader got;
  std::memcpy(&got, p, sizeof got);
  const CkptHeader want = ckpt_header(d);
  if (std::memcmp(&got, &want, sizeof got) != 0)
    return fail(PLACE_EINVAL, "the checkpoint was taken on a handle of another design, grid or "
                "parameters (header mismatch)");
  p += pad8(sizeof got);
  // the copy's queued work ends before its state is replaced
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpyAsync(d.cs + copy, p, sizeof(CopyState), cudaMemcpyHostToDevice, h->stream));
  p += pad8(sizeof(CopyState));
  for (const CkptArray &a : ckpt_arrays(d, copy)) {
    CK(cudaMemcpyAsync(a.dev, p, a.bytes, cudaMemcpyHostToDevice, h->stream));
    p += pad8(a.bytes);
  }
  h->k0_pending = true;  // the loaded state may be at k = 0
  CK(cudaStreamSynchronize(h->stream));
  return check_dev_err(h);
}

int place_get_stretched_map(place_t *h, int32_t copy, int64_t *map) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (!map) return fail(PLACE_EINVAL, "null output");
  if (!h->d.Ms) return fail(PLACE_EINVAL, "density stretching is off for this handle");
  CK(cudaMemcpyAsync(map, h->d.Ms + (size_t)copy * h->d.G, sizeof(int64_t) * h->d.G,
                     cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PLACE_OK;
}

int place_get_positions(place_t *h, int32_t copy, float *x, float *y) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  const size_t C = h->d.n_cells;
  return copy_out_xy(h, h->d.xy + copy * C, x, y);
}

int place_get_fillers(place_t *h, int32_t copy, float *x, float *y, int32_t cap, int32_t *n) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (cap < 0) return fail(PLACE_EINVAL, "cap < 0");
  const Dev &d = h->d;
  if (n) *n = d.n_fill;
  const int m = std::min(cap, d.n_fill);
  if (m > 0 && (x || y)) {
    launch_unpack_xy(d.px_tmp, d.py_tmp, d.xy + (size_t)copy * d.n_cells + d.n_real, m, h->stream);
    CKL();
    if (x) CK(cudaMemcpyAsync(x, d.px_tmp, sizeof(float) * m, cudaMemcpyDefault, h->stream));
    if (y) CK(cudaMemcpyAsync(y, d.py_tmp, sizeof(float) * m, cudaMemcpyDefault, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return PLACE_OK;
}

int place_set_fillers(place_t *h, int32_t copy, const float *x, const float *y) {
  int rc = check_copy(h, copy, true);
  if (rc) return rc;
  const Dev &d = h->d;
  if (d.n_fill == 0) return PLACE_OK;
  if (!x || !y) return fail(PLACE_EINVAL, "null positions");
  const int c0 = copy < 0 ? 0 : copy, n = copy < 0 ? d.K : 1;
  CK(cudaMemcpyAsync(d.px_tmp, x, sizeof(float) * d.n_fill, cudaMemcpyDefault, h->stream));
  CK(cudaMemcpyAsync(d.py_tmp, y, sizeof(float) * d.n_fill, cudaMemcpyDefault, h->stream));
  for (int c = c0; c < c0 + n; ++c)
    launch_pack_xy(d.xy + (size_t)c * d.n_cells + d.n_real, d.px_tmp, d.py_tmp, d.n_fill, h->stream);
  return enqueue_reset(h, c0, n);
}

int place_device_views(place_t *h, int32_t copy, float **x, float **y) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (!x || !y) return fail(PLACE_EINVAL, "null output");
  float *base = reinterpret_cast<float *>(h->d.xy + (size_t)copy * h->d.n_cells);
  *x = base;
  *y = base + 1;
  return PLACE_OK;
}

int place_set_positions(place_t *h, int32_t copy, const float *x, const float *y) {
  int rc = check_copy(h, copy, true);
  if (rc) return rc;
  if (!x || !y) return fail(PLACE_EINVAL, "null positions");
  const size_t C = h->d.n_cells, Mv = h->d.n_real;
  int c0 = copy < 0 ? 0 : copy, n = copy < 0 ? h->d.K : 1;
  CK(cudaMemcpyAsync(h->d.px_tmp, x, sizeof(float) * Mv, cudaMemcpyDefault, h->stream));
  CK(cudaMemcpyAsync(h->d.py_tmp, y, sizeof(float) * Mv, cudaMemcpyDefault, h->stream));
  for (int c = c0; c < c0 + n; ++c) launch_pack_xy(h->d.xy + c * C, h->d.px_tmp, h->d.py_tmp, (int)Mv, h->stream);
  return enqueue_reset(h, c0, n);
}

int place_eval_wirelength(place_t *h, int32_t copy, float gamma, double *wl, float *gx, float *gy) {
  NvtxRange nvtx_("place_eval_wirelength");
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (!(gamma > 0.f)) return fail(PLACE_EINVAL, "gamma must be > 0");
  Dev &d = h->d;
  float *gdev = reinterpret_cast<float *>(d.scal + (size_t)copy * S_COUNT + S_G2);
  CK(cudaMemcpyAsync(gdev, &gamma, sizeof(float), cudaMemcpyHostToDevice, h->stream));
  // the sums of a stopped copy's last WA pass may not have been consumed
  CK(cudaMemsetAsync(d.gacc + (size_t)copy * d.n_mov, 0, sizeof(unsigned long long) * d.n_mov, h->stream));
  launch_wa(d, copy, 1, 1, gdev, h->stream);
  launch_cell_grad(d, copy, 1, 1, h->stream);
  launch_reduce_slot(d, S_WL, d.wa_blocks_total, copy, 1, h->stream);
  CKL();
  const size_t Mo = d.n_mov, Mv = d.n_real;  // per-copy stride, the design's movable cells
  if (gx) CK(cudaMemcpyAsync(gx, d.gwx + copy * Mo, sizeof(float) * Mv, cudaMemcpyDefault, h->stream));
  if (gy) CK(cudaMemcpyAsync(gy, d.gwy + copy * Mo, sizeof(float) * Mv, cudaMemcpyDefault, h->stream));
  double v = 0;
  CK(cudaMemcpyAsync(&v, d.scal + (size_t)copy * S_COUNT + S_WL, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if ((rc = check_dev_err(h))) return rc;
  if (wl) *wl = v;
  return PLACE_OK;
}

}  // extern "C"

namespace {

int density_at(place_t *h, int copy) {
  Dev &d = h->d;
  CK(cudaMemsetAsync(d.M + (size_t)copy * d.Gm, 0, sizeof(unsigned long long) * d.Gm, h->stream));
  launch_scatter(d, copy, 1, 1, h->stream);
  launch_density_finish(d, copy, 1, FIN_EVAL, h->stream);
  CKL();
  return PLACE_OK;
}

}  // namespace

extern "C" {

int place_eval_density(place_t *h, int32_t copy, int64_t *map, double *overflow) {
  NvtxRange nvtx_("place_eval_density");
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  Dev &d = h->d;
  if ((rc = density_at(h, copy))) return rc;
  if (map) CK(cudaMemcpyAsync(map, d.M + (size_t)copy * d.Gm, sizeof(int64_t) * d.G, cudaMemcpyDefault, h->stream));
  double s = 0;
  CK(cudaMemcpyAsync(&s, d.scal + (size_t)copy * S_COUNT + S_TAU, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (overflow) *overflow = s;
  return PLACE_OK;
}

int place_get_fixed_map(place_t *h, int64_t *map) {
  if (!h || !map) return fail(PLACE_EINVAL, "null argument");
  CK(cudaMemcpyAsync(map, h->d.Fmap, sizeof(int64_t) * h->d.G, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PLACE_OK;
}

int place_eval_field(place_t *h, int32_t copy, float *psi, float *ex, float *ey) {
  NvtxRange nvtx_("place_eval_field");
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  Dev &d = h->d;
  if ((rc = density_at(h, copy))) return rc;
  launch_spectral(d, copy, 1, 1, 1, h->stream);
  CKL();
  const size_t G = d.G;
  const float *E = d.E + (size_t)copy * 3 * G;
  if (ex) CK(cudaMemcpyAsync(ex, E, sizeof(float) * G, cudaMemcpyDefault, h->stream));
  if (ey) CK(cudaMemcpyAsync(ey, E + G, sizeof(float) * G, cudaMemcpyDefault, h->stream));
  if (psi) CK(cudaMemcpyAsync(psi, E + 2 * G, sizeof(float) * G, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_dev_err(h);
}

int place_eval_density_grad(place_t *h, int32_t copy, float *gx, float *gy) {
  NvtxRange nvtx_("place_eval_density_grad");
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  Dev &d = h->d;
  if ((rc = density_at(h, copy))) return rc;
  launch_spectral(d, copy, 1, 0, 1, h->stream);
  launch_cell_grad(d, copy, 1, 1, h->stream);
  CKL();
  const size_t Mo = d.n_mov, Mv = d.n_real;  // per-copy stride, the design's movable cells
  if (gx) CK(cudaMemcpyAsync(gx, d.gdx + copy * Mo, sizeof(float) * Mv, cudaMemcpyDefault, h->stream));
  if (gy) CK(cudaMemcpyAsync(gy, d.gdy + copy * Mo, sizeof(float) * Mv, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_dev_err(h);
}

int place_eval_hpwl_overflow(place_t *h, double *hpwl, double *overflow) {
  NvtxRange nvtx_("place_eval_hpwl_overflow");
  if (!h) return fail(PLACE_EINVAL, "null handle");
  Dev &d = h->d;
  const int K = d.K;
  launch_hpwl64(d, 0, K, h->stream);
  launch_reduce_slot(d, S_HP64, d.cell_blocks + 2 * std::max(d.cell_blocks / 2, 1), 0, K, h->stream);
  CK(cudaMemsetAsync(d.M, 0, sizeof(unsigned long long) * (size_t)d.Gm * K, h->stream));
  launch_scatter(d, 0, K, 1, h->stream);
  launch_density_finish(d, 0, K, FIN_EVAL, h->stream);
  CKL();
  std::vector<double> sc((size_t)K * S_COUNT);
  CK(cudaMemcpyAsync(sc.data(), d.scal, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (int rc = check_dev_err(h)) return rc;
  for (int c = 0; c < K; ++c) {
    if (hpwl) hpwl[c] = sc[(size_t)c * S_COUNT + S_HP64];
    if (overflow) overflow[c] = sc[(size_t)c * S_COUNT + S_TAU];
  }
  return PLACE_OK;
}

int place_perturb(place_t *h, int32_t op, float p, uint64_t seed, int32_t copy) {
  NvtxRange nvtx_("place_perturb");
  int rc = check_copy(h, copy, true);
  if (rc) return rc;
  if (op == PLACE_WIREMASK) {
    const int c0 = copy < 0 ? 0 : copy, n = copy < 0 ? h->d.K : 1;
    if (!h->wm_order.empty()) {
      if ((rc = ensure_wiremask(h))) return rc;
      cudaGraphExec_t &ex = h->wm_graphs[std::make_pair(c0, n)];
      if (!ex) {
        // the tables are uploaded on h->stream; the capture stream waits for them
        CK(cudaEventRecord(h->ev_fork, h->stream));
        CK(cudaStreamWaitEvent(h->cap, h->ev_fork, 0));
        CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        launch_wiremask(h->d, h->wm, h->wm_ptr.data(), c0, n, h->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          ex = nullptr;
          h->wm_graphs.erase(std::make_pair(c0, n));
          return fail(PLACE_ECUDA, "WireMask graph: %s", cudaGetErrorString(e));
        }
      }
      CK(cudaGraphLaunch(ex, h->stream));
    }
    return enqueue_reset(h, c0, n);
  }
  if (op != PLACE_SHUFFLE_MACRO && op != PLACE_SHUFFLE_ALL) return fail(PLACE_EINVAL, "unknown perturbation op %d", op);
  if (!(p >= 0.f && p <= 1.f)) return fail(PLACE_EINVAL, "p must be in [0, 1]");
  Dev &d = h->d;
  const int ncand = op == PLACE_SHUFFLE_ALL ? h->n_cand_all : h->n_cand_macro;
  int k = (int)std::floor((double)p * ncand + 0.5);
  k = std::max(0, std::min(k, ncand));
  int c0 = copy < 0 ? 0 : copy, n = copy < 0 ? d.K : 1;
  for (int c = c0; c < c0 + n; ++c) {
    uint64_t sd = copy < 0 ? seed + (uint64_t)c : seed;
    if (k > 0) {
      launch_shuffle(d, c, op, p, sd, h->stream);
      launch_shuffle_finish(d, c, k, h->stream);
      CKL();
    }
  }
  return enqueue_reset(h, c0, n);
}

int place_hybro(place_t *h, int32_t n_rounds, int32_t op, float p, uint64_t seed, float tau_target,
                double *best_hpwl, double *best_overflow, int32_t *best_round) {
  NvtxRange nvtx_("place_hybro");
  if (!h) return fail(PLACE_EINVAL, "null handle");
  if (n_rounds < 0) return fail(PLACE_EINVAL, "n_rounds < 0");
  Dev &d = h->d;
  const int K = d.K;
  const size_t C = d.n_cells;
  std::vector<double> bh(K, 0.0), bt(K, 0.0), hp(K), tau(K);
  std::vector<int> br(K, -1), conv(K);
  const int nrec = n_rounds + 1;
  h->round_hpwl.assign((size_t)K * nrec, 0.0);
  h->round_tau.assign((size_t)K * nrec, 0.0);
  h->n_round_records = 0;
  for (int r = 0; r <= n_rounds; ++r) {
    NvtxRange nvtx_round("hybro round");
    // place every copy until it stops (converged or max_iters)
    for (;;) {
      int rc = place_step(h, 32, conv.data());
      if (rc) return rc;
      bool all = true;
      for (int c = 0; c < K; ++c) all = all && conv[c];
      if (all) break;
    }
    int rc = place_eval_hpwl_overflow(h, hp.data(), tau.data());
    if (rc) return rc;
    for (int c = 0; c < K; ++c) {
      h->round_hpwl[(size_t)c * nrec + r] = hp[c];
      h->round_tau[(size_t)c * nrec + r] = tau[c];
    }
    h->n_round_records = r + 1;
    for (int c = 0; c < K; ++c) {
      bool better = br[c] < 0;
      if (!better) {
        int fa = tau[c] <= tau_target ? 0 : 1, fb = bt[c] <= tau_target ? 0 : 1;
        better = fa != fb ? fa < fb : (hp[c] != bh[c] ? hp[c] < bh[c] : tau[c] < bt[c]);
      }
      if (better) {
        bh[c] = hp[c]; bt[c] = tau[c]; br[c] = r;
        CK(cudaMemcpyAsync(d.bxy + c * C, d.xy + c * C, sizeof(float2) * C, cudaMemcpyDeviceToDevice, h->stream));
      }
    }
    if (r < n_rounds) {
      for (int c = 0; c < K; ++c) {
        int rc2 = place_perturb(h, op, p, seed + (uint64_t)r * K + c, c);
        if (rc2) return rc2;
      }
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  for (int c = 0; c < K; ++c) {
    if (best_hpwl) best_hpwl[c] = bh[c];
    if (best_overflow) best_overflow[c] = bt[c];
    if (best_round) best_round[c] = br[c];
  }
  h->best_hpwl = bh; h->best_tau = bt; h->best_round = br;
  return PLACE_OK;
}

int place_get_best_positions(place_t *h, int32_t copy, float *x, float *y) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (h->best_round.empty()) return fail(PLACE_EINVAL, "place_hybro has not run on this handle");
  const size_t C = h->d.n_cells;
  return copy_out_xy(h, h->d.bxy + copy * C, x, y);
}

int place_get_hybro_rounds(place_t *h, int32_t copy, double *hpwl, double *overflow, int32_t cap,
                           int32_t *n_records) {
  int rc = check_copy(h, copy, false);
  if (rc) return rc;
  if (h->n_round_records <= 0) return fail(PLACE_EINVAL, "place_hybro has not run on this handle");
  if (cap < 0) return fail(PLACE_EINVAL, "cap < 0");
  const int n = h->n_round_records;
  const size_t stride = h->round_hpwl.size() / (size_t)h->d.K;
  for (int r = 0; r < std::min(n, (int)cap); ++r) {
    if (hpwl) hpwl[r] = h->round_hpwl[(size_t)copy * stride + r];
    if (overflow) overflow[r] = h->round_tau[(size_t)copy * stride + r];
  }
  if (n_records) *n_records = n;
  return PLACE_OK;
}

}  // extern "C"

extern "C" int place_estimate_device_bytes(const place_netlist *nl, const place_die *die,
                                           const place_bins *bins, const place_params *params,
                                           int64_t *bytes) {
  if (!nl || !bins || !bytes) return fail(PLACE_EINVAL, "null argument");
  place_params prm;
  if (params) prm = *params; else place_default_params(&prm);
  if (nl->n_cells <= 0 || nl->n_pins < 0 || nl->n_nets < 0 || bins->nx <= 0 || bins->ny <= 0 ||
      prm.n_copies < 1)
    return fail(PLACE_EINVAL, "bad sizes");
  // filler cells: counted exactly as place_create counts them (the die is
  // needed for that; without it, or without the netlist's arrays, none)
  long long nf = 0;
  if (prm.fillers && die && nl->w && nl->h && nl->x0 && nl->y0 && die->xh > die->xl &&
      die->yh > die->yl) {
    double total_area = 0.0;
    for (int i = 0; i < nl->n_cells; ++i) total_area += (double)nl->w[i] * (double)nl->h[i];
    const int F = choose_frac_bits(die, total_area);
    if (F >= 0) {
      const double s = std::ldexp(1.0, F);
      unsigned __int128 mov_area_q = 0;
      for (int i = 0; i < nl->n_movable; ++i)
        mov_area_q += (unsigned __int128)(unsigned long long)std::nearbyint((double)nl->w[i] * s) *
                      (unsigned __int128)(unsigned long long)std::nearbyint((double)nl->h[i] * s);
      nf = plan_fillers(nl, die, bins, F, mov_area_q).n;
    }
  }
  // the layout of place_create with upper bounds for the sizes that depend on
  // the netlist's contents (pins on movable cells, reduction slots)
  Dev d{};
  d.K = prm.n_copies;
  d.n_cells = nl->n_cells + (int)nf; d.n_mov = nl->n_movable + (int)nf;
  d.n_real = nl->n_movable; d.n_fill = (int)nf;
  d.n_nets = nl->n_nets; d.n_pins = nl->n_pins;
  d.nx = bins->nx; d.ny = bins->ny; d.G = bins->nx * bins->ny;
  d.Gm = nf ? 2 * d.G : d.G;
  d.has_net_w = nl->net_w ? 1 : 0;
  prm.dct_mode = resolve_dct_mode(prm.dct_mode, bins->nx, bins->ny);
  d.tc = prm.dct_mode == PLACE_DCT_BF16X3 ? 1 : 0;
  d.bfly = use_fold(d.tc, prm.dct_fold, bins->nx, bins->ny);
  d.prm = prm;
  const int cb = std::max(1, std::min((d.n_mov + kThreads - 1) / kThreads, kMaxCellBlocks));
  const int bb = std::max(1, std::min((d.G + kThreads - 1) / kThreads, kMaxCellBlocks));
  d.nb_red = std::max(std::max(2 * cb + 2, bb), 4 * kMaxCellBlocks + kMaxBigNetBlocks);
  int sn = 2;
  while (sn < d.n_cells) sn <<= 1;
  d.sort_n = sn;
  Arena a;
  layout(d, a, d.K);
  *bytes = (int64_t)(a.off + 256);
  return PLACE_OK;
}

namespace hp {

// Launch n iterations on the handle's stream, then copy the copies' stopped
// flags into host memory (pinned, [K]) and record `ev`; never blocks.
int step_async(place_t *h, int n, int *stopped_host, cudaEvent_t ev) {
  if (n > 0) {
    int rc = ensure_graph(h);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) CK(launch_iter(h));
  }
  for (int c = 0; c < h->d.K; ++c)
    CK(cudaMemcpyAsync(stopped_host + c, &h->d.cs[c].stopped, sizeof(int), cudaMemcpyDeviceToHost,
                       h->stream));
  CK(cudaEventRecord(ev, h->stream));
  return PLACE_OK;
}

// Positions of copy 0 of `src` into every copy of `dst` (same design),
// device to device on dst's stream after src's work; resets dst's optimiser.
int copy_positions(place_t *dst, place_t *src, cudaEvent_t src_done) {
  if (dst->d.n_cells != src->d.n_cells) return fail(PLACE_EINVAL, "designs differ");
  CK(cudaEventRecord(src_done, src->stream));
  CK(cudaStreamWaitEvent(dst->stream, src_done, 0));
  const size_t C = dst->d.n_cells;
  for (int c = 0; c < dst->d.K; ++c)
    CK(cudaMemcpyAsync(dst->d.xy + c * C, src->d.xy, sizeof(float2) * C, cudaMemcpyDeviceToDevice,
                       dst->stream));
  return enqueue_reset(dst, 0, dst->d.K);
}

cudaStream_t handle_stream(place_t *h) { return h->stream; }

// Copy 0's positions into a device buffer (stream-ordered on h's stream).
int save_xy(place_t *h, float2 *dst) {
  CK(cudaMemcpyAsync(dst, h->d.xy, sizeof(float2) * h->d.n_cells, cudaMemcpyDeviceToDevice,
                     h->stream));
  return PLACE_OK;
}

// Every copy of h takes the positions in `src` (device); resets the optimiser.
int load_xy(place_t *h, const float2 *src) {
  const size_t C = h->d.n_cells;
  for (int c = 0; c < h->d.K; ++c)
    CK(cudaMemcpyAsync(h->d.xy + c * C, src, sizeof(float2) * C, cudaMemcpyDeviceToDevice,
                       h->stream));
  return enqueue_reset(h, 0, h->d.K);
}

}  // namespace hp
