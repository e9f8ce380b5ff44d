// place_overflow_noalloc: the density map and overflow of a placement,
// computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc when they need this number: a host
// framework whose memory pool owns all device memory during a step, a
// real-time or embedded service that forbids allocation after start-up, or
// a callback that must not trigger the implicit device synchronisation an
// allocation can cause.  For them this entry point keeps its scratch (the
// 64-bit density map, the reduction partials and the movable-area sum) in one
// file-scope `static __device__` array of fixed size, allocated with the
// module and held by every GPU that loads the library until the process
// exits.  The caller passes the inputs and the outputs; nothing else is
// needed.
//
// Limits and sharing: at most PLACE_NOALLOC_MAX_BINS bins.  Every call uses
// the same array, which keeps the last call's contents; each call clears the
// map, the area sum, the flags and the reduction counter before use.  Calls
// whose work overlaps on the GPU (two streams, or two host threads) race on
// the array and give wrong results: serialise them.  The device address of
// the array is looked up once per device with cudaGetSymbolAddress on the
// first call made with that device current; make that first call before any
// stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <mutex>

#include "../../include/hybro_place.h"
#include "common.cuh"

namespace hp {
void set_last_error(const char *msg);  // api.cu
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 1024;  // blocks of the per-bin pass (partials slots)
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  unsigned long long map[PLACE_NOALLOC_MAX_BINS];
  unsigned long long part[kNaBlocks * 2];
  // cleared by every call (one memset from area_lo to the end)
  unsigned long long area_lo, area_hi;  // exact sum of W H over the cells (128 bits)
  unsigned int counter;                 // last-block counter of the finish pass
  int bad;                              // a cell size outside [1, 2^31) units
  int dbg[4];                           // failed index check (bounds-checking build)
};

static __device__ __align__(256) NoAllocScratch g_scratch;

NoAllocScratch *g_dev_ptr[kMaxDevices] = {};
std::mutex g_setup_mu;

int na_fail(int code, const char *fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);  // reported by place_last_error()
  return code;
}

struct NaGrid {
  float scale;
  long long XL, YL, BW, BH;
  int nx, ny;
  long long t_mant;
  int t_shift;
};

// Quantised sizes W = rint(w 2^F), H = rint(h 2^F) (w 2^F is exact in FP32),
// the cells' exact overlaps added to the map, and the exact sum of W H.  A
// size outside [1, 2^31) raises the scratch's `bad` flag and the cell is
// skipped (the handle path rejects such a cell at create).
__global__ void __launch_bounds__(kNaThreads)
    k_na_scatter(NoAllocScratch *s, const float *x, const float *y, const float *w, const float *h,
                 int n, NaGrid g) {
  __shared__ u128 sm[32];
  u128 area = 0;
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float ws = w[i] * g.scale, hs = h[i] * g.scale;
    // also false for NaN sizes
    if (!(ws >= 0.5f && ws < 2147483647.0f && hs >= 0.5f && hs < 2147483647.0f)) {
      bad = true;
      continue;
    }
    const long long W = __float2ll_rn(ws), H = __float2ll_rn(hs);
    if (W < 1 || H < 1 || W > 2147483647LL || H > 2147483647LL) {
      bad = true;
      continue;
    }
    area += (u128)(unsigned long long)(W * H);
    QRect r = qrect(x[i], y[i], (int)W, (int)H, g.scale, g.XL, g.YL, g.BW, g.BH, g.nx, g.ny);
    for (int ix = r.ix0; ix <= r.ix1; ++ix) {
      long long ox = overlap1(r.X, r.W, g.XL + (long long)ix * g.BW, g.BW);
      if (ox == 0) continue;
      for (int iy = r.iy0; iy <= r.iy1; ++iy) {
        long long oy = overlap1(r.Y, r.H, g.YL + (long long)iy * g.BH, g.BH);
        if (oy == 0) continue;
        const long long b = (long long)ix * g.ny + iy;
        if (!HP_IN(s->dbg, b, (long long)g.nx * g.ny, BS_NOALLOC_BIN)) continue;
        atomicAdd(&s->map[b], (unsigned long long)(ox * oy));
      }
    }
  }
  if (bad) s->bad = 1;
  const u128 a = block_sum_u128<kNaThreads>(area, sm);
  if (threadIdx.x == 0 && a != 0) {
    // 128-bit accumulation from two 64-bit atomics with the carry propagated
    const unsigned long long lo = (unsigned long long)a, hi = (unsigned long long)(a >> 64);
    const unsigned long long old = atomicAdd(&s->area_lo, lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&s->area_hi, hi + carry);
  }
}

__global__ void __launch_bounds__(kNaThreads)
    k_na_finish(NoAllocScratch *s, const long long *fixed_map, NaGrid g, double *overflow,
                long long *map_out) {
  __shared__ u128 sm[32];
  __shared__ int flag;
  const int G = g.nx * g.ny;
  const long long abin = g.BW * g.BH;
  u128 acc = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < G; b += gridDim.x * blockDim.x) {
    const long long m = (long long)s->map[b];
    const long long f = fixed_map ? fixed_map[b] : 0ll;
    const __int128 e = ((__int128)m << g.t_shift) - (__int128)g.t_mant * (__int128)(abin - f);
    if (e > 0) acc += (u128)e;
    if (map_out) map_out[b] = m;
  }
  u128 r = block_sum_u128<kNaThreads>(acc, sm);
  if (threadIdx.x == 0) {
    s->part[2 * blockIdx.x] = (unsigned long long)r;
    s->part[2 * blockIdx.x + 1] = (unsigned long long)(r >> 64);
  }
  if (!arrive_last(&s->counter, &flag)) return;
  u128 v = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
    v += ((u128)s->part[2 * i + 1] << 64) | s->part[2 * i];
  v = block_sum_u128<kNaThreads>(v, sm);
  if (threadIdx.x == 0) {
    // the movable area in units of 2^-2F; the map's entries stay below it, so
    // beyond 2^62 (or with a rejected cell) the map itself is not trusted
    const unsigned long long lo = *(volatile unsigned long long *)&s->area_lo;
    const unsigned long long hi = *(volatile unsigned long long *)&s->area_hi;
    const int bad = *(volatile int *)&s->bad || *(volatile int *)&s->dbg[2];
    if (bad || hi != 0 || lo >= (1ull << 62)) {
      *overflow = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
    } else {
      const double amov = lo > 0 ? (double)lo : 1.0;
      *overflow = ldexp(u128_to_double(v), -g.t_shift) / amov;
    }
    s->counter = 0u;
  }
}

// Device address of the static scratch for the current device (set-up on
// the first call with that device current).
int scratch_ptr(NoAllocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(PLACE_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(PLACE_EINVAL, "device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_dev_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(PLACE_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                     cudaGetErrorString(e));
    g_dev_ptr[dev] = static_cast<NoAllocScratch *>(p);
  }
  *out = g_dev_ptr[dev];
  return PLACE_OK;
}

bool dyadic(double v, double s) {
  const double q = v * s;
  return std::isfinite(q) && std::floor(q) == q;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int place_overflow_noalloc(const float *x, const float *y, const float *w,
                                      const float *h, int32_t n_movable, const place_die *die,
                                      const place_bins *bins, int32_t frac_bits,
                                      const int64_t *fixed_map, double *overflow,
                                      int64_t *map_out, void *stream) {
  if (!die || !bins || !overflow) return na_fail(PLACE_EINVAL, "null die, bins or overflow");
  if (n_movable < 0) return na_fail(PLACE_EINVAL, "n_movable < 0");
  if (n_movable > 0 && (!x || !y || !w || !h)) return na_fail(PLACE_EINVAL, "null cell array");
  const int nx = bins->nx, ny = bins->ny;
  if (nx <= 0 || ny <= 0) return na_fail(PLACE_EINVAL, "bins must be positive, got %dx%d", nx, ny);
  if ((long long)nx * ny > PLACE_NOALLOC_MAX_BINS)
    return na_fail(PLACE_EINVAL, "%dx%d bins exceed the static scratch of %d bins", nx, ny,
                   PLACE_NOALLOC_MAX_BINS);
  if (frac_bits < 0 || frac_bits > 24) return na_fail(PLACE_EINVAL, "frac_bits must be in [0, 24]");
  if (!(bins->target_density > 0.f)) return na_fail(PLACE_EINVAL, "target density must be > 0");
  if (!(die->xh > die->xl) || !(die->yh > die->yl)) return na_fail(PLACE_EINVAL, "empty die");
  const double s = std::ldexp(1.0, frac_bits);
  // the extent rule of the handle's resolution F: every coordinate of the die
  // and its extent, times 2^F, below 2^30 (keeps the bin arithmetic in range)
  const double ext = std::fmax(std::fmax(std::fmax(std::fabs(die->xl), std::fabs(die->xh)),
                                         std::fmax(std::fabs(die->yl), std::fabs(die->yh))),
                               std::fmax(die->xh - die->xl, die->yh - die->yl));
  if (!(ext * s < std::ldexp(1.0, 30)))
    return na_fail(PLACE_ERANGE, "frac_bits %d is too fine for this die: extent 2^F must stay "
                   "below 2^30", frac_bits);
  const double bw = (die->xh - die->xl) / nx, bh = (die->yh - die->yl) / ny;
  if (!dyadic(die->xl, s) || !dyadic(die->yl, s) || !dyadic(bw, s) || !dyadic(bh, s) ||
      !(bw * s >= 1.0) || !(bh * s >= 1.0))
    return na_fail(PLACE_EINVAL, "die origin and bin size must be multiples of 2^-%d", frac_bits);
  NaGrid g;
  g.scale = (float)s;
  g.XL = (long long)(die->xl * s); g.YL = (long long)(die->yl * s);
  g.BW = (long long)(bw * s); g.BH = (long long)(bh * s);
  g.nx = nx; g.ny = ny;
  int e2 = 0;
  const double f = std::frexp((double)bins->target_density, &e2);
  g.t_mant = (long long)std::ldexp(f, 24);
  g.t_shift = 24 - e2;
  if (g.t_shift < 0 || g.t_shift > 60) return na_fail(PLACE_EINVAL, "target density out of range");

  NoAllocScratch *sp = nullptr;
  int rc = scratch_ptr(&sp);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(sp->map, 0, sizeof(unsigned long long) * (size_t)nx * ny, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(&sp->area_lo, 0,
                        sizeof(NoAllocScratch) - offsetof(NoAllocScratch, area_lo), st);
  if (e != cudaSuccess) return na_fail(PLACE_ECUDA, "clearing the scratch: %s", cudaGetErrorString(e));
  if (n_movable > 0) {
    int blocks = (n_movable + kNaThreads - 1) / kNaThreads;
    if (blocks > 4096) blocks = 4096;
    k_na_scatter<<<blocks, kNaThreads, 0, st>>>(sp, x, y, w, h, n_movable, g);
  }
  int fb = (nx * ny + kNaThreads - 1) / kNaThreads;
  if (fb > kNaBlocks) fb = kNaBlocks;
  k_na_finish<<<fb, kNaThreads, 0, st>>>(sp, reinterpret_cast<const long long *>(fixed_map), g,
                                         overflow, reinterpret_cast<long long *>(map_out));
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(PLACE_ECUDA, "launch: %s", cudaGetErrorString(e));
  return PLACE_OK;
}
