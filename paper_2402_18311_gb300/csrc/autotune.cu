// Create-time autotuner: tile shapes and kernel variants chosen by timing
// candidates on the handle's own device state.
//
// Three knobs, none of which changes a result bit (the candidates compute the
// same integers, or the same FP32 operations per output element):
//  * the tile width N of each tensor-core GEMM stage of the spectral solve
//    (128: fewer CTAs, more reuse per CTA; 64: twice the CTAs for grids that
//    would leave SMs idle) and whether a stage with few tiles splits its
//    contraction over two CTAs per tile;
//  * how many pins of a net above 256 pins the big-net WA kernel keeps in
//    shared memory (more pins cached, fewer blocks resident per SM);
//  * on how many graph branches the WA degree classes run (one chain, or two
//    or three chains side by side, so that the tails of the classes with few
//    long blocks overlap the classes with many short ones).
//  These run beside other kernels of the iteration (the wirelength branch and
//  the density/spectral branch share the GPU), so they are timed as whole
//  iterations of the captured graph, every candidate from the same start;
//  * the two effective-bin thresholds at which the density scatter switches
//    from merging a warp's shared bins to the shared-memory table and from
//    the table to direct atomics.  The scatter's cost depends on how
//    concentrated the cells are, which changes during a placement, so the
//    three ways are timed on centred Gaussian clouds of the design's own cells
//    at widths that span the phases of a placement, and the thresholds are
//    put where the fastest way changes.
// Results are cached in the process per shape (grid, copies, cell, pin and
// degree magnitudes), so a job server creating many similar handles tunes
// once per shape.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace hp {
namespace {

struct Key {
  int nx, ny, K, tc, lg_mov, lg_pins, lg_deg, stretch, gemm_bn, gemm_split, cap, scat, wa_streams,
      fold;
  bool operator<(const Key &o) const {
    return std::tie(nx, ny, K, tc, lg_mov, lg_pins, lg_deg, stretch, gemm_bn, gemm_split, cap,
                    scat, wa_streams, fold) <
           std::tie(o.nx, o.ny, o.K, o.tc, o.lg_mov, o.lg_pins, o.lg_deg, o.stretch, o.gemm_bn,
                    o.gemm_split, o.cap, o.scat, o.wa_streams, o.fold);
  }
};

std::mutex g_mu;
std::map<Key, TuneOut> g_cache;

constexpr int kTuneIters = 16;  // graph iterations timed per candidate run
// A candidate replaces the incumbent (the first, the fixed rule's choice)
// only when it is faster by more than this fraction: the graph-level timing
// varies by about 1% from run to run.
constexpr float kTuneMargin = 0.015f;

// Best of two timed runs of the iteration graph (ms per iteration).
float time_graph(const TuneHooks &hk) {
  const float a = hk.time_iters(hk.ctx, kTuneIters);
  if (a < 0.f) return a;
  const float b = hk.time_iters(hk.ctx, kTuneIters);
  return b < 0.f ? b : std::min(a, b);
}

int lg2(long long v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

// Copy 0's movable cells as a centred Gaussian cloud, standard deviation
// (sx, sy) per axis, clamped into the die.  Counter-based: cell i's normals
// come from a SplitMix64 hash of (seed, i) through Box-Muller, so the cloud is
// the same on every call.
__global__ void k_tune_cloud(Dev d, float sx, float sy, unsigned long long seed) {
  const float cx = 0.5f * (d.fxl + d.fxh), cy = 0.5f * (d.fyl + d.fyh);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u1 = ((float)(z >> 40) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = (float)((z >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
    const float r = sqrtf(-2.0f * logf(u1));
    const float gx = r * cosf(6.2831853f * u2), gy = r * sinf(6.2831853f * u2);
    const float w = d.w[i], h = d.h[i];
    const float x = fminf(fmaxf(cx + sx * gx - 0.5f * w, d.fxl), d.fxh - w);
    const float y = fminf(fmaxf(cy + sy * gy - 0.5f * h, d.fyl), d.fyh - h);
    d.xy[i] = make_float2(x, y);
  }
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  // Smallest device time of `reps` runs of f (ms); `pre` runs before each,
  // outside the timed span.  Negative on a CUDA error.
  template <typename F, typename G>
  float best(int reps, F f, G pre) {
    float m = 1e30f;
    for (int r = 0; r < reps; ++r) {
      pre();
      cudaEventRecord(a, st);
      f();
      cudaEventRecord(b, st);
      if (cudaEventSynchronize(b) != cudaSuccess) return -1.f;
      float t = 0.f;
      cudaEventElapsedTime(&t, a, b);
      m = std::min(m, t);
    }
    return cudaGetLastError() == cudaSuccess ? m : -1.f;
  }
};

}  // namespace

int autotune(Dev &d, int max_deg, cudaStream_t st, const TuneHooks &hk, TuneOut *out) {
  const auto t0 = std::chrono::steady_clock::now();
  const Key key{d.nx,           d.ny,           d.K,           d.tc,
                lg2(d.n_mov),   lg2(d.n_pins),  lg2(max_deg),  d.prm.stretch,
                d.prm.gemm_bn,  d.prm.gemm_split, d.prm.wa_big_cap, d.prm.scatter_mode,
                d.prm.wa_streams, d.bfly};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second;
      out->cached = 1;
      out->ms = 0.0;
      for (int s = 0; s < 4; ++s) {
        d.tc_bn[s] = out->bn[s];
        d.tc_split[s] = out->split[s];
      }
      d.wa_big_cap = out->cap;
      d.wa_streams = out->wa_streams;
      d.scat_t1 = out->t1;
      d.scat_t2 = out->t2;
      return d.tc ? hk.encode_maps(hk.ctx) : 0;
    }
  }
  Timer tm(st);

  // 1. tile width of the tensor-core GEMM stages.  The solve shares the GPU
  // with the wirelength kernels on the iteration's second stream, so the
  // objective is the whole iteration: each candidate is timed over iterations
  // of the captured graph from the same start.
  if (d.tc && (d.prm.gemm_bn == 0 || d.prm.gemm_split == 0)) {
    // tile width per stage, and split-K on the stages with few tiles (the
    // first two, or all four, where the workspace allows it)
    struct Cand { int bn[4], split[4]; };
    const Cand all[7] = {{{128, 128, 128, 128}, {1, 1, 1, 1}}, {{128, 128, 128, 128}, {2, 2, 1, 1}},
                         {{128, 128, 128, 128}, {1, 1, 2, 2}}, {{128, 128, 128, 128}, {2, 2, 2, 2}},
                         {{64, 64, 128, 128}, {1, 1, 1, 1}}, {{128, 128, 64, 64}, {1, 1, 1, 1}},
                         {{64, 64, 64, 64}, {1, 1, 1, 1}}};
    std::vector<Cand> cand;
    for (const Cand &c0 : all) {
      Cand c = c0;
      for (int s = 0; s < 4; ++s) {
        if (d.prm.gemm_bn) c.bn[s] = d.prm.gemm_bn;
        if (d.prm.gemm_split) c.split[s] = d.prm.gemm_split;
        if (!d.tc_split_ok[s] || c.bn[s] != 128) c.split[s] = 1;
      }
      bool dup = false;
      for (const Cand &e : cand)
        dup = dup || (std::equal(e.bn, e.bn + 4, c.bn) && std::equal(e.split, e.split + 4, c.split));
      if (!dup) cand.push_back(c);
    }
    // the fixed rule's choice first: it stays unless another is clearly faster
    Cand rule;
    for (int s = 0; s < 4; ++s) {
      rule.bn[s] = d.tc_bn[s];
      rule.split[s] = d.tc_split[s];
    }
    cand.insert(cand.begin(), rule);
    float best_t = 1e30f;
    size_t best_c = 0;
    for (size_t c = 0; c < cand.size(); ++c) {
      if (c > 0 && std::equal(rule.bn, rule.bn + 4, cand[c].bn) &&
          std::equal(rule.split, rule.split + 4, cand[c].split))
        continue;
      for (int s = 0; s < 4; ++s) {
        d.tc_bn[s] = cand[c].bn[s];
        d.tc_split[s] = cand[c].split[s];
      }
      if (int rc = hk.encode_maps(hk.ctx)) return rc;
      const float t = time_graph(hk);
      if (t < 0.f) return PLACE_ECUDA;
      if (c == 0 || t < best_t * (1.f - kTuneMargin)) {
        best_t = t;
        best_c = c;
      }
    }
    for (int s = 0; s < 4; ++s) {
      d.tc_bn[s] = cand[best_c].bn[s];
      d.tc_split[s] = cand[best_c].split[s];
    }
    if (int rc = hk.encode_maps(hk.ctx)) return rc;
  }

  // 2. shared-memory cap of the big-net WA kernel, the same way
  if (d.prm.wa_big_cap == 0 && d.n_cls > 4 && d.wa_blocks[4] > 0) {
    std::vector<int> cand{d.wa_big_cap};  // the fixed rule's cap first
    for (int c : {1024, 2048, 3072, 4096, 6144})
      if (c < max_deg && c != d.wa_big_cap) cand.push_back(c);
    if (std::min(max_deg, 6144) != d.wa_big_cap) cand.push_back(std::min(max_deg, 6144));
    if (wa_prepare(*std::max_element(cand.begin(), cand.end()))) return PLACE_ECUDA;
    float best_t = 1e30f;
    int best_c = d.wa_big_cap;
    for (size_t i = 0; i < cand.size(); ++i) {
      d.wa_big_cap = cand[i];
      const float t = time_graph(hk);
      if (t < 0.f) return PLACE_ECUDA;
      if (i == 0 || t < best_t * (1.f - kTuneMargin)) {
        best_t = t;
        best_c = cand[i];
      }
    }
    d.wa_big_cap = best_c;
  }

  // 2b. graph branches of the WA classes, the same way
  if (d.prm.wa_streams == 0 && d.n_cls > 1) {
    const int rule = d.wa_streams;
    float best_t = 1e30f;
    int best_n = rule;
    const int cand[3] = {rule, rule == 2 ? 1 : 2, rule == 3 ? 1 : 3};
    for (int i = 0; i < 3; ++i) {
      d.wa_streams = cand[i];
      const float t = time_graph(hk);
      if (t < 0.f) return PLACE_ECUDA;
      if (i == 0 || t < best_t * (1.f - kTuneMargin)) {
        best_t = t;
        best_n = cand[i];
      }
    }
    d.wa_streams = best_n;
  }

  // 3. the scatter's thresholds, from clouds of increasing width (the
  // scatter's cost depends on the phase, which one start cannot show)
  if (d.prm.scatter_mode < 0 && d.n_mov > 0) {
    constexpr int nl = 10;
    std::vector<double> neff(nl);
    std::vector<float> tmode[3];
    for (auto &v : tmode) v.assign(nl, 0.f);
    const size_t mbytes = sizeof(unsigned long long) * (size_t)d.Gm;
    const int blocks = std::max(1, std::min((d.n_mov + kThreads - 1) / kThreads, kMaxCellBlocks));
    for (int l = 0; l < nl; ++l) {
      const float width = 0.0004f * std::pow(2.0f, (float)l);  // 0.0004 .. 0.2 of the die
      k_tune_cloud<<<blocks, kThreads, 0, st>>>(d, width * (d.fxh - d.fxl), width * (d.fyh - d.fyl),
                                                0x5EEDull + l);
      // the cloud's effective number of bins, from one density pass
      cudaMemsetAsync(d.M, 0, mbytes, st);
      d.scat_force = SCAT_MERGED;
      launch_scatter_main(d, 0, 1, 1, st);
      launch_density_finish(d, 0, 1, FIN_RESET, st);
      CopyState cs;
      if (cudaMemcpyAsync(&cs, d.cs, sizeof cs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return PLACE_ECUDA;
      neff[l] = std::max(cs.n_eff, 1.0);
      for (int m = SCAT_MERGED; m <= SCAT_DIRECT; ++m) {
        // direct atomics on a very dense cloud serialise badly; one run shows it
        const int reps = (m == SCAT_DIRECT && l < 3) ? 1 : 3;
        d.scat_force = m;
        const float t = tm.best(reps, [&] { launch_scatter_main(d, 0, 1, 1, st); },
                                [&] { cudaMemsetAsync(d.M, 0, mbytes, st); });
        if (t < 0.f) return PLACE_ECUDA;
        tmode[m][l] = t;
      }
    }
    d.scat_force = -1;
    // where one way stops being slower than another: the zero of their time
    // difference, interpolated linearly in log n_eff between the clouds
    auto crossing = [&](int a, int b) {
      for (int l = 0; l < nl; ++l) {
        const float dl = tmode[a][l] - tmode[b][l];
        if (dl <= 0.f) continue;  // a still faster here
        if (l == 0) return 0.5 * neff[0];
        const float dp = tmode[a][l - 1] - tmode[b][l - 1];
        const double f = dp < 0.f ? (double)(-dp) / ((double)dl - (double)dp) : 0.0;
        return std::exp(std::log(neff[l - 1]) + f * (std::log(neff[l]) - std::log(neff[l - 1])));
      }
      return 1e300;
    };
    const double t1 = crossing(SCAT_MERGED, SCAT_TABLE);
    const double t2 = crossing(SCAT_TABLE, SCAT_DIRECT);
    d.scat_t1 = std::min(t1, t2);
    d.scat_t2 = t2;
  }

  out->cached = 0;
  for (int s = 0; s < 4; ++s) {
    out->bn[s] = d.tc_bn[s];
    out->split[s] = d.tc_split[s];
  }
  out->cap = d.wa_big_cap;
  out->wa_streams = d.wa_streams;
  out->t1 = d.scat_t1;
  out->t2 = d.scat_t2;
  out->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = *out;
  return 0;
}

}  // namespace hp
