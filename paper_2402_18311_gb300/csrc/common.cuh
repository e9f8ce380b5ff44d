// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hp {

// ---- bounds-checking build ----------------------------------------------
// Index sites of the bounds-checking build (HP_IN below); names for the
// error message are in api.cu (bound_site_name).
enum BoundSite {
  BS_NONE = 0,
  BS_WA_PIN,        // a net's CSR pin range in the WA kernels
  BS_WA_CELL,       // a pin's cell in the WA kernels
  BS_HPWL_PIN,      // a net's CSR pin range in the exact HPWL kernels
  BS_HPWL_CELL,     // a pin's cell there
  BS_GRAD_CELL,     // the cell a pin's gradient is added to
  BS_MAP_BIN,       // a density-map entry written by a scatter
  BS_FIELD_BIN,     // a field entry read by the cell-gradient gather
  BS_TILE_ROW,      // a GEMM output row or column
  BS_WM_NET,        // WireMask: a net or pin index
  BS_WM_CELL,       // WireMask: a cell index
  BS_WM_BIN,        // WireMask: a bin of the mask or the profile
  BS_PERM,          // a Shuffle permutation or candidate index
  BS_NOALLOC_BIN,   // place_overflow_noalloc: a map entry
  BS_COUNT
};

// Built with -DPLACE_DEBUG_BOUNDS, HP_IN(err, i, n, site) tests 0 <= i < n for
// an index about to be used (a CSR offset, a cell, a bin, a tile row); a failed test records the first failing site and its index in
// err[2] and err[3] (the host reports them as PLACE_EINTERNAL) and yields
// false, and the caller then skips the access or uses index 0 instead.  In
// the normal build HP_IN is the constant true and its arguments are not
// evaluated.  The sites are the BoundSite values.
#ifdef PLACE_DEBUG_BOUNDS
static __device__ __noinline__ void bound_fail(int *err, int site, long long i) {
  if (atomicCAS(err + 2, 0, site) == 0)
    atomicExch(err + 3, (int)(i < -2147483647LL ? -2147483647LL : (i > 2147483647LL ? 2147483647LL : i)));
}
#define HP_IN(err, i, n, site)                                              \
  (((long long)(i) >= 0 && (long long)(i) < (long long)(n))                 \
       ? true                                                               \
       : (::hp::bound_fail((err), (site), (long long)(i)), false))
#else
#define HP_IN(err, i, n, site) true
#endif
// An index that fails HP_IN is replaced by 0 (a valid element) so that the
// code after it needs no second branch.
#define HP_FIX(err, var, n, site) \
  do {                            \
    if (!HP_IN(err, var, n, site)) (var) = 0; \
  } while (0)

__device__ __forceinline__ long long floordiv_ll(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// Deterministic block sum of one double per thread (fixed shuffle/smem tree);
// the result is valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (l < NT / 32) ? sm[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// Deterministic block sum of floats (fixed tree); valid in thread 0.
template <int NT>
__device__ __forceinline__ float block_sum_f(float v, float *sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x < 32) {
    r = (l < NT / 32) ? sm[l] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// Block sum of one float per thread, compensated: every addition of the
// shuffle tree is an error-free two-sum (the rounding error of s = a + b is
// (a - (s - b')) + (b - b') with b' = s - a, exact in FP32), and the errors
// travel with the sums, so the result has about FP64 accuracy while all the
// arithmetic stays on the FP32 pipes (GB300's FP64 rate is a small fraction
// of its FP32 rate).  Returns (sum, correction) folded into a double, valid
// in thread 0.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
template <int NT>
__device__ __forceinline__ double block_sum_fc(float v, float2 *sm) {
  float c = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float w = __shfl_xor_sync(0xffffffffu, v, o), wc = __shfl_xor_sync(0xffffffffu, c, o);
    float e;
    two_sum(v, w, v, e);
    c = __fadd_rn(c, __fadd_rn(wc, e));
  }
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[wi] = make_float2(v, c);
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    const float2 p = (l < NT / 32) ? sm[l] : make_float2(0.f, 0.f);
    v = p.x;
    c = p.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float w = __shfl_xor_sync(0xffffffffu, v, o), wc = __shfl_xor_sync(0xffffffffu, c, o);
      float e;
      two_sum(v, w, v, e);
      c = __fadd_rn(c, __fadd_rn(wc, e));
    }
    r = (double)v + (double)c;
  }
  return r;
}

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, o);
  hi = __shfl_xor_sync(0xffffffffu, hi, o);
  return ((u128)hi << 64) | lo;
}

// Exact block sum of unsigned 128-bit integers; valid in thread 0.
template <int NT>
__device__ __forceinline__ u128 block_sum_u128(u128 v, u128 *sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  u128 r = 0;
  if (threadIdx.x < 32) {
    r = (l < NT / 32) ? sm[l] : (u128)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += shfl_xor_u128(r, o);
  }
  return r;
}

__device__ __forceinline__ double u128_to_double(u128 v) {
  return (double)(unsigned long long)(v >> 64) * 18446744073709551616.0 +
         (double)(unsigned long long)v;
}

// Last-block pattern: every block has published its partials; returns true
// (in all threads) for the block that arrives last, which then reduces the
// partials in a fixed order and resets the counter.
__device__ __forceinline__ bool arrive_last(unsigned int *ctr, int *sm_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(ctr, 1u);
    *sm_flag = (prev == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *sm_flag != 0;
  if (last) __threadfence();
  return last;
}

// floor(a / b) for b > 0 and |a| below 2^40: a float estimate of the
// quotient, then one exact integer correction in each direction (the
// estimate is off by at most one for these magnitudes).
__device__ __forceinline__ long long floordiv_est(long long a, long long b, float inv_b) {
  long long q = (long long)floorf((float)a * inv_b);
  if (q * b > a) --q;
  if ((q + 1) * b <= a) ++q;
  return q;
}

// Quantised rectangle of a cell and the clipped bin range it touches.
struct QRect {
  long long X, Y, W, H;
  int ix0, ix1, iy0, iy1;
};

__device__ __forceinline__ QRect qrect(float x, float y, int W, int H, float scale, long long XL,
                                       long long YL, long long BW, long long BH, int nx, int ny) {
  QRect r;
  // x * 2^F is exact in FP32; rounding to the nearest integer, ties to even
  // non-finite or huge coordinates saturate far outside the die (empty range)
  const float lim = 4.0e18f;
  float xs = x * scale, ys = y * scale;
  xs = (xs == xs) ? fminf(fmaxf(xs, -lim), lim) : -lim;
  ys = (ys == ys) ? fminf(fmaxf(ys, -lim), lim) : -lim;
  r.X = __float2ll_rn(xs);
  r.Y = __float2ll_rn(ys);
  r.W = W;
  r.H = H;
  // offsets far outside the die are clipped to one bin beyond it first, which
  // leaves the clipped range unchanged and keeps the quotients small
  const long long lox = -BW, hix = (long long)(nx + 1) * BW;
  const long long loy = -BH, hiy = (long long)(ny + 1) * BH;
  long long ax0 = r.X - XL, ax1 = r.X + r.W - 1 - XL, ay0 = r.Y - YL, ay1 = r.Y + r.H - 1 - YL;
  ax0 = ax0 < lox ? lox : (ax0 > hix ? hix : ax0);
  ax1 = ax1 < lox ? lox : (ax1 > hix ? hix : ax1);
  ay0 = ay0 < loy ? loy : (ay0 > hiy ? hiy : ay0);
  ay1 = ay1 < loy ? loy : (ay1 > hiy ? hiy : ay1);
  const float ibw = 1.0f / (float)BW, ibh = 1.0f / (float)BH;
  long long a0 = floordiv_est(ax0, BW, ibw), a1 = floordiv_est(ax1, BW, ibw);
  long long b0 = floordiv_est(ay0, BH, ibh), b1 = floordiv_est(ay1, BH, ibh);
  // clip to the grid in 64 bits before narrowing; an empty range (lo > hi)
  // results for rectangles outside the die or non-finite coordinates
  a0 = a0 < 0 ? 0 : (a0 > nx ? nx : a0);
  a1 = a1 >= nx ? nx - 1 : (a1 < -1 ? -1 : a1);
  b0 = b0 < 0 ? 0 : (b0 > ny ? ny : b0);
  b1 = b1 >= ny ? ny - 1 : (b1 < -1 ? -1 : b1);
  r.ix0 = (int)a0;
  r.ix1 = (int)a1;
  r.iy0 = (int)b0;
  r.iy1 = (int)b1;
  return r;
}

__device__ __forceinline__ long long overlap1(long long lo, long long size, long long b0,
                                              long long step) {
  long long hi = lo + size, bh = b0 + step;
  long long o = (hi < bh ? hi : bh) - (lo > b0 ? lo : b0);
  return o > 0 ? o : 0;
}

// The same rectangle in 32-bit integers, relative to the die's lower-left
// corner.  The fixed-point resolution keeps nx * BW and ny * BH below 2^30,
// and the edges are clipped to two bins beyond the die, which changes no
// overlap with any bin; so every edge, quotient and overlap below fits int32
// and only the area product needs 64 bits.
struct QRect32 {
  int x0, x1, y0, y1;      // edges [x0, x1) x [y0, y1), relative and clipped
  int ix0, ix1, iy0, iy1;  // clipped bin range (empty when ix0 > ix1)
};

__device__ __forceinline__ int clip_to_int(long long v, long long lo, long long hi) {
  return (int)(v < lo ? lo : (v > hi ? hi : v));
}

// floor(a / b) for b > 0 and |a| + 2b < 2^31: a float estimate of the
// quotient (off by at most one here), then one exact correction each way.
__device__ __forceinline__ int floordiv32(int a, int b, float inv_b) {
  int q = (int)floorf((float)a * inv_b);
  if (q * b > a) --q;
  if ((q + 1) * b <= a) ++q;
  return q;
}

__device__ __forceinline__ QRect32 qrect32(float x, float y, int W, int H, float scale,
                                           long long XL, long long YL, int BW, int BH, int nx,
                                           int ny, float inv_bw, float inv_bh) {
  // x * 2^F is exact in FP32; rounding to the nearest integer, ties to even;
  // non-finite or huge coordinates saturate far outside the die
  const float lim = 4.0e18f;
  float xs = x * scale, ys = y * scale;
  xs = (xs == xs) ? fminf(fmaxf(xs, -lim), lim) : -lim;
  ys = (ys == ys) ? fminf(fmaxf(ys, -lim), lim) : -lim;
  const long long X = __float2ll_rn(xs) - XL, Y = __float2ll_rn(ys) - YL;
  const long long lox = -2LL * BW, hix = (long long)(nx + 2) * BW;
  const long long loy = -2LL * BH, hiy = (long long)(ny + 2) * BH;
  QRect32 r;
  r.x0 = clip_to_int(X, lox, hix);
  r.x1 = clip_to_int(X + W, lox, hix);
  r.y0 = clip_to_int(Y, loy, hiy);
  r.y1 = clip_to_int(Y + H, loy, hiy);
  r.ix0 = max(floordiv32(r.x0, BW, inv_bw), 0);
  r.ix1 = min(floordiv32(r.x1 - 1, BW, inv_bw), nx - 1);
  r.iy0 = max(floordiv32(r.y0, BH, inv_bh), 0);
  r.iy1 = min(floordiv32(r.y1 - 1, BH, inv_bh), ny - 1);
  return r;
}

// Overlap of the relative interval [lo, hi) with bin k of width b.
__device__ __forceinline__ int overlap32(int lo, int hi, int k, int b) {
  const int b0 = k * b;
  const int o = min(hi, b0 + b) - max(lo, b0);
  return o > 0 ? o : 0;
}

}  // namespace hp
