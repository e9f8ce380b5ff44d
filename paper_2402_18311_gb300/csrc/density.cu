// Electrostatic density: exact overlap-area bin map in 64-bit fixed point and
// its conversion to bin density and overflow.
//
// The density D of Eq. 1/2 is the ePlace electrostatic density the paper
// cites.  Reading: coordinates quantised to multiples of 2^-F (x * 2^F is
// exact in FP32, rounded to the nearest integer with ties to even), movable
// map M_b = sum_i overlap(cell_i, bin_b) as int64 in units of 2^-2F,
// overflow tau = sum_b max(0, M_b - t (A_b - F_b)) / A_mov and bin density
// rho_b = (M_b + t F_b) / A_b.  Integer addition is associative, so the map
// is bit-exact and independent of the order in which cells are added.  The
// overflow sum is exact too: with t = m 2^-s (m < 2^24), every bin's excess
// times 2^s is an integer below 2^100, summed in 128-bit integers.
#include "common.cuh"
#include "internal.cuh"

namespace hp {

constexpr int kHash = 2048;  // shared-memory aggregation table entries

// Adds one (bin, area) contribution to the block's shared-memory table, or to
// the global map when its slot is taken (bounded linear probing).  lim: the
// map's length (checked in the bounds-checking build only).
__device__ __forceinline__ void hash_add(int *keys, unsigned long long *vals,
                                         unsigned long long *M, int b,
                                         unsigned long long a, int *err, int lim) {
  if (!HP_IN(err, b, lim, BS_MAP_BIN)) return;
  unsigned int hsh = ((unsigned int)b * 2654435761u) >> (32 - 11);
#pragma unroll 1
  for (int probe = 0; probe < 2; ++probe) {
    int k = keys[hsh];  // plain read first: no atomic when the bin is already there
    if (k == -1) k = atomicCAS(&keys[hsh], -1, b);
    if (k == -1 || k == b) {
      atomicAdd(&vals[hsh], a);
      return;
    }
    hsh = (hsh + 1) & (kHash - 1);
  }
  atomicAdd(&M[b], a);
}

// Exact sum of 64-bit values over the lanes in `mask` (all of which call
// this with the same mask): three 21-bit limbs are summed with the 32-bit
// warp reduction, which cannot overflow for 32 lanes.  The scatter calls it
// with the full mask only.
__device__ __forceinline__ unsigned long long group_sum_u64(unsigned int mask,
                                                            unsigned long long a) {
  const unsigned int l0 = (unsigned int)(a & 0x1FFFFF);
  const unsigned int l1 = (unsigned int)((a >> 21) & 0x1FFFFF);
  const unsigned int l2 = (unsigned int)(a >> 42);
  const unsigned long long s0 = __reduce_add_sync(mask, l0);
  const unsigned long long s1 = __reduce_add_sync(mask, l1);
  const unsigned long long s2 = __reduce_add_sync(mask, l2);
  return s0 + (s1 << 21) + (s2 << 42);
}

// Exact warp sum of values below 2^42: two 21-bit limbs (the second below
// 2^21, so each limb's sum over 32 lanes stays below 2^26).
__device__ __forceinline__ unsigned long long warp_sum_u42(unsigned long long a) {
  const unsigned long long s0 = __reduce_add_sync(0xffffffffu, (unsigned int)(a & 0x1FFFFF));
  const unsigned long long s1 = __reduce_add_sync(0xffffffffu, (unsigned int)(a >> 21));
  return s0 + (s1 << 21);
}

// The scatter's three ways (ScatterMode) are chosen per copy from the
// effective number of occupied bins of the previous density pass, n_eff =
// (sum M)^2 / sum M^2, against the handle's thresholds d.scat_t1 < d.scat_t2
// (set at create, by the autotuner when it runs).

// In the merged path, a warp slot whose lanes form more shared-bin groups
// than this adds every term to the block table instead.  Measured on the
// 2.1M-cell design, density stage at iterations 5 / 155: 0.112 / 0.144 ms
// with per-group reductions always, 0.100 / 0.126 with this cut-off (8: no
// change; always adding directly: 0.151 / 0.064, but 0.271 at iteration 55).
constexpr int kMaxMergeGroups = 4;

// Cells are processed grid-stride, a warp at a time, in one of three ways,
// chosen per copy from how concentrated the previous density pass was:
//  * SCAT_MERGED, very dense (the centred start of a placement, where
//    millions of cells share a few bins): each cell touches at most 2 x 2
//    bins when it is no larger than a bin; the warp visits those four slots
//    in lock-step, lanes that hit the same bin are merged with a match/reduce
//    (exact integer sums), and one lane per distinct bin adds the total to a
//    shared-memory hash table that is flushed with one 64-bit atomic per
//    distinct bin;
//  * SCAT_TABLE, concentrated (the middle of a placement, tens to a few
//    thousand effective bins): every lane adds each term to the block's
//    shared-memory table without the match, which costs more than the
//    shared-memory conflicts it would remove once the lanes of a warp rarely
//    share a bin;
//  * SCAT_DIRECT, spread: each lane adds its overlaps straight to the map.
// Larger cells add their remaining bins through the table in the first two
// ways.  Every way adds the same integers, so the map is the same.
__global__ void __launch_bounds__(kThreads) k_scatter(Dev d, int copy0, int eval) {
  __shared__ int keys[kHash];
  __shared__ unsigned long long vals[kHash];
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  for (int i = threadIdx.x; i < kHash; i += blockDim.x) {
    keys[i] = -1;
    vals[i] = 0ull;
  }
  __syncthreads();
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  unsigned long long *M = d.M + (size_t)c * d.Gm;
  const int stride = gridDim.x * blockDim.x;
  const double n_eff = d.cs[c].n_eff;
  // map index of cell i's bin b: b for a movable cell, G + b for a filler
  // (the fillers' map follows the movable one)
  const int mode = d.scat_force >= 0 ? d.scat_force
                                     : (n_eff < d.scat_t1 ? SCAT_MERGED
                                                          : (n_eff < d.scat_t2 ? SCAT_TABLE : SCAT_DIRECT));
  if (mode == SCAT_DIRECT) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += stride) {
      const int mo = i < d.n_real ? 0 : d.G;
      const float2 v = xy[i];
      const QRect32 r = qrect32(v.x, v.y, d.Wq[i], d.Hq[i], d.scale, d.XL, d.YL, d.BW32, d.BH32,
                                d.nx, d.ny, d.ibw_q, d.ibh_q);
      for (int ix = r.ix0; ix <= r.ix1; ++ix) {
        const int ox = overlap32(r.x0, r.x1, ix, d.BW32);
        if (ox == 0) continue;
        for (int iy = r.iy0; iy <= r.iy1; ++iy) {
          const int oy = overlap32(r.y0, r.y1, iy, d.BH32);
          if (oy == 0) continue;
          const int b = mo + ix * d.ny + iy;
          if (HP_IN(d.err, b, d.Gm, BS_MAP_BIN))
            atomicAdd(&M[b], (unsigned long long)((long long)ox * oy));
        }
      }
    }
    return;
  }
  if (mode == SCAT_TABLE) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += stride) {
      const int mo = i < d.n_real ? 0 : d.G;
      const float2 v = xy[i];
      const QRect32 r = qrect32(v.x, v.y, d.Wq[i], d.Hq[i], d.scale, d.XL, d.YL, d.BW32, d.BH32,
                                d.nx, d.ny, d.ibw_q, d.ibh_q);
      for (int ix = r.ix0; ix <= r.ix1; ++ix) {
        const int ox = overlap32(r.x0, r.x1, ix, d.BW32);
        if (ox == 0) continue;
        for (int iy = r.iy0; iy <= r.iy1; ++iy) {
          const int oy = overlap32(r.y0, r.y1, iy, d.BH32);
          if (oy == 0) continue;
          hash_add(keys, vals, M, mo + ix * d.ny + iy, (unsigned long long)((long long)ox * oy),
                   d.err, d.Gm);
        }
      }
    }
  } else {
  // one cell's overlap with one bin is at most the bin area
  const bool two_limbs = (double)d.BW * (double)d.BH < 4398046511104.0;  // 2^42
  // warp-uniform trip count
  for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < d.n_mov; i0 += stride) {
    const int i = i0 + (threadIdx.x & 31);
    const bool valid = i < d.n_mov;
    const int mo = i < d.n_real ? 0 : d.G;
    QRect32 r;
    if (valid) {
      const float2 v = xy[i];
      r = qrect32(v.x, v.y, d.Wq[i], d.Hq[i], d.scale, d.XL, d.YL, d.BW32, d.BH32, d.nx, d.ny,
                  d.ibw_q, d.ibh_q);
    } else {
      r.x0 = r.x1 = r.y0 = r.y1 = 0;
      r.ix0 = r.iy0 = 0;
      r.ix1 = r.iy1 = -1;
    }
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
      const int ix = r.ix0 + (sl & 1), iy = r.iy0 + (sl >> 1);
      int b = -1;
      unsigned long long a = 0ull;
      if (ix <= r.ix1 && iy <= r.iy1) {
        const int ox = overlap32(r.x0, r.x1, ix, d.BW32);
        const int oy = overlap32(r.y0, r.y1, iy, d.BH32);
        a = (unsigned long long)((long long)ox * oy);
        if (a != 0ull) b = mo + ix * d.ny + iy;
      }
      // one full-warp reduction per bin shared by several lanes (a per-group
      // mask would serialise the groups inside every reduction); each
      // group's lowest lane keeps the total, then all of them add at once:
      // alone on its bin straight to the map, shared through the block table
      const unsigned int mask = __match_any_sync(0xffffffffu, b);
      const int lane = threadIdx.x & 31;
      const bool lead = b >= 0 && lane == __ffs(mask) - 1;
      const bool shared = __popc(mask) > 1;
      unsigned int groups = __ballot_sync(0xffffffffu, lead && shared);
      if (__popc(groups) > kMaxMergeGroups) {
        // many small groups: one reduction per group would cost more than
        // the few same-address conflicts of adding every term to the table
        if (b >= 0) hash_add(keys, vals, M, b, a, d.err, d.Gm);
        continue;
      }
      unsigned long long tot = a;
      while (groups) {
        const int l = __ffs(groups) - 1;
        groups &= groups - 1;
        const int key = __shfl_sync(0xffffffffu, b, l);
        const unsigned long long mine = b == key ? a : 0ull;
        const unsigned long long t =
            two_limbs ? warp_sum_u42(mine) : group_sum_u64(0xffffffffu, mine);
        if (lane == l) tot = t;
      }
      if (lead) {
        if (shared)
          hash_add(keys, vals, M, b, tot, d.err, d.Gm);
        else if (HP_IN(d.err, b, d.Gm, BS_MAP_BIN))
          atomicAdd(&M[b], tot);
      }
    }
    // bins beyond the first 2 x 2 (cells larger than a bin)
    if (valid && (r.ix1 - r.ix0 > 1 || r.iy1 - r.iy0 > 1)) {
      for (int ix = r.ix0; ix <= r.ix1; ++ix) {
        const int ox = overlap32(r.x0, r.x1, ix, d.BW32);
        if (ox == 0) continue;
        for (int iy = r.iy0; iy <= r.iy1; ++iy) {
          if (ix - r.ix0 <= 1 && iy - r.iy0 <= 1) continue;  // done above
          const int oy = overlap32(r.y0, r.y1, iy, d.BH32);
          if (oy == 0) continue;
          hash_add(keys, vals, M, mo + ix * d.ny + iy, (unsigned long long)((long long)ox * oy),
                   d.err, d.Gm);
        }
      }
    }
  }
  }  // SCAT_MERGED
  __syncthreads();
  for (int i = threadIdx.x; i < kHash; i += blockDim.x) {
    int k = keys[i];
    if (k >= 0) atomicAdd(&M[k], vals[i]);
  }
}

// Density stretching (ePlace local smoothing): the map that drives the field
// when it is on.  Every movable cell enters as its stretched rectangle
// (create-time offsets and sizes in d.st) and each (cell, bin) term is
// floor(ov R / 2^31) with the cell's fixed-point scale R = d.sR[i] <= 2^31:
// ov = q 2^31 + r gives q R + floor(r R / 2^31), exact in 64 bits.  Terms go
// through the block's shared-memory table (the centred start is dense).
__global__ void __launch_bounds__(kThreads) k_scatter_stretch(Dev d, int copy0, int eval) {
  __shared__ int keys[kHash];
  __shared__ unsigned long long vals[kHash];
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  for (int i = threadIdx.x; i < kHash; i += blockDim.x) {
    keys[i] = -1;
    vals[i] = 0ull;
  }
  __syncthreads();
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  unsigned long long *M = d.Ms + (size_t)c * d.G;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    const float2 v = xy[i];
    const int4 st = d.st[i];  // {x shift, y shift, stretched W, stretched H}
    const unsigned long long R = d.sR[i];
    const QRect32 r = qrect32(v.x, v.y, st.z, st.w, d.scale, d.XL + st.x, d.YL + st.y, d.BW32,
                              d.BH32, d.nx, d.ny, d.ibw_q, d.ibh_q);
    for (int ix = r.ix0; ix <= r.ix1; ++ix) {
      const int ox = overlap32(r.x0, r.x1, ix, d.BW32);
      if (ox == 0) continue;
      for (int iy = r.iy0; iy <= r.iy1; ++iy) {
        const int oy = overlap32(r.y0, r.y1, iy, d.BH32);
        if (oy == 0) continue;
        const unsigned long long ov = (unsigned long long)((long long)ox * oy);
        const unsigned long long t = (ov >> 31) * R + (((ov & 0x7fffffffull) * R) >> 31);
        if (t) hash_add(keys, vals, M, ix * d.ny + iy, t, d.err, d.G);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHash; i += blockDim.x) {
    int k = keys[i];
    if (k >= 0) atomicAdd(&M[k], vals[i]);
  }
}

// Same map for an arbitrary cell range (the fixed cells, once at create).
__global__ void __launch_bounds__(kThreads)
    k_scatter_range(Dev d, const float2 *xy, int n0, int n1, unsigned long long *out) {
  for (int i = n0 + blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) {
    const float2 v = xy[i];
    const QRect32 r = qrect32(v.x, v.y, d.Wq[i], d.Hq[i], d.scale, d.XL, d.YL, d.BW32, d.BH32,
                              d.nx, d.ny, d.ibw_q, d.ibh_q);
    for (int ix = r.ix0; ix <= r.ix1; ++ix) {
      const int ox = overlap32(r.x0, r.x1, ix, d.BW32);
      if (ox == 0) continue;
      for (int iy = r.iy0; iy <= r.iy1; ++iy) {
        const int oy = overlap32(r.y0, r.y1, iy, d.BH32);
        if (oy == 0) continue;
        const int b = ix * d.ny + iy;
        if (HP_IN(d.err, b, d.G, BS_MAP_BIN))
          atomicAdd(&out[b], (unsigned long long)((long long)ox * oy));
      }
    }
  }
}

// A nonnegative 64-bit integer as FP32 from its two 32-bit halves (two fast
// conversions and one FMA instead of the multi-instruction 64-bit one; the
// result may differ from the correctly rounded one in the last bit).
__device__ __forceinline__ float u64_to_float(unsigned long long v) {
  return fmaf((float)(unsigned int)(v >> 32), 4294967296.0f, (float)(unsigned int)v);
}

// Excess contribution of one bin: bins without fixed cells are counted into
// (m_over, n_over) and closed after the loop; the others are summed exactly
// in 128 bits.
__device__ __forceinline__ void bin_excess(const Dev &d, unsigned long long m, long long f, u128 tA,
                                           u128 &acc, unsigned long long &m_over,
                                           unsigned int &n_over) {
  if (f == 0) {
    if (m > d.tA_floor) {
      m_over += m;
      ++n_over;
    }
  } else {
    // excess * 2^s = m 2^s + t_mant F - t_mant A: exact in unsigned 128
    // bits (below 2^124, and valid when overlapping fixed cells make F > A)
    u128 lhs = (u128)m << d.t_shift;
    lhs += (u128)(unsigned long long)d.t_mant * (u128)(unsigned long long)f;
    if (lhs > tA) acc += lhs - tA;
  }
}

// One pair of bins (2 b2, 2 b2 + 1): their excess into the sums and rho.
template <bool STRETCH>
__device__ __forceinline__ float2 finish_pair(const Dev &d, int c, int b2, const ulonglong2 *M2,
                                              const ulonglong2 *Mf2, const longlong2 *F2,
                                              u128 tA, float inv_a, float tf, u128 &acc,
                                              unsigned long long &m_over, unsigned int &n_over,
                                              float &q2) {
  const ulonglong2 m = M2[b2];
  const longlong2 f = F2[b2];
  float mq0 = u64_to_float(m.x) * inv_a, mq1 = u64_to_float(m.y) * inv_a;
  if (Mf2) {
    const ulonglong2 mf = Mf2[b2];
    mq0 = u64_to_float(m.x + mf.x) * inv_a;
    mq1 = u64_to_float(m.y + mf.y) * inv_a;
  }
  q2 = fmaf(mq0, mq0, q2);
  q2 = fmaf(mq1, mq1, q2);
  bin_excess(d, m.x, f.x, tA, acc, m_over, n_over);
  bin_excess(d, m.y, f.y, tA, acc, m_over, n_over);
  float mf0 = mq0, mf1 = mq1;
  if constexpr (STRETCH) {
    const ulonglong2 ms = reinterpret_cast<const ulonglong2 *>(d.Ms + (size_t)c * d.G)[b2];
    mf0 = u64_to_float(ms.x) * inv_a;
    mf1 = u64_to_float(ms.y) * inv_a;
  }
  return make_float2(fmaf(tf, u64_to_float((unsigned long long)f.x) * inv_a, mf0),
                     fmaf(tf, u64_to_float((unsigned long long)f.y) * inv_a, mf1));
}

__device__ __forceinline__ void store_bf16_pair(__nv_bfloat16 *hp, __nv_bfloat16 *lp, size_t b2,
                                                float v0, float v1) {
  const __nv_bfloat162 hi = __floats2bfloat162_rn(v0, v1);
  const __nv_bfloat162 lo = __floats2bfloat162_rn(v0 - __low2float(hi), v1 - __high2float(hi));
  reinterpret_cast<__nv_bfloat162 *>(hp)[b2] = hi;
  reinterpret_cast<__nv_bfloat162 *>(lp)[b2] = lo;
}

// Per bin: exact overflow excess and rho in FP32; the last block of each copy
// reduces the excess and, by mode, records the overflow as the iteration's
// tau (with the stop test), as an evaluation result, or as the reset value
// tau_{-1} that sets the first gamma.  STRETCH: rho comes from the
// stretched map (density stretching on); the overflow always from M.  Two
// bins per thread and step (G is even): 16-byte loads and paired bf16
// conversions and stores.  FOLD (the even/odd split of the tensor-core
// solve): four bins per step, (x, y), (x, y+1) and their mirrors
// (x, ny-1-y), (x, ny-2-y), and rho leaves as the sums rho_y + rho_{ny-1-y}
// at y and the differences at ny/2 + y (y < ny/2).
template <bool STRETCH, bool FOLD>
__global__ void __launch_bounds__(kThreads) k_density_finish(Dev d, int copy0, int mode) {
  __shared__ u128 sm[32];
  __shared__ float smf[32];
  __shared__ int flag;
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  CopyState *cs = d.cs + c;
  if (mode == FIN_ITER && cs->stopped) return;
  const ulonglong2 *M2 = reinterpret_cast<const ulonglong2 *>(d.M + (size_t)c * d.Gm);
  // with fillers their map (following M) joins rho and the concentration
  const ulonglong2 *Mf2 = d.n_fill ? M2 + (d.G >> 1) : nullptr;
  const longlong2 *F2 = reinterpret_cast<const longlong2 *>(d.Fmap);
  const u128 tA = ((u128)d.tA_hi << 64) | d.tA_lo;  // t_mant * A_bin
  const float inv_a = (float)(1.0 / d.abin_q);
  const float tf = (float)d.t;
  u128 acc = 0;
  // bins without fixed cells: their excess times 2^s is m 2^s - t_mant A,
  // positive exactly when m > floor(t_mant A / 2^s); the sum over those bins
  // is 2^s (sum of m) - count * t_mant A, formed once after the loop (the
  // sum of m stays below the movable area, below 2^62)
  unsigned long long m_over = 0ull;
  unsigned int n_over = 0u;
  float q2 = 0.f;
  if constexpr (FOLD) {
    __nv_bfloat16 *rh = d.rho_h + (size_t)c * d.G, *rl = d.rho_l + (size_t)c * d.G;
    const int q4 = d.ny >> 2, nq = d.G >> 2, hy = d.ny >> 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += gridDim.x * blockDim.x) {
      const int x = t / q4, y = 2 * (t - x * q4);  // y even, below ny/2
      const int row = x * d.ny;
      const float2 a = finish_pair<STRETCH>(d, c, (row + y) >> 1, M2, Mf2, F2, tA, inv_a, tf, acc,
                                            m_over, n_over, q2);
      // bins ny-2-y and ny-1-y
      const float2 b = finish_pair<STRETCH>(d, c, (row + d.ny - 2 - y) >> 1, M2, Mf2, F2, tA,
                                            inv_a, tf, acc, m_over, n_over, q2);
      store_bf16_pair(rh, rl, (size_t)(row + y) >> 1, __fadd_rn(a.x, b.y), __fadd_rn(a.y, b.x));
      store_bf16_pair(rh, rl, (size_t)(row + hy + y) >> 1, __fsub_rn(a.x, b.y),
                      __fsub_rn(a.y, b.x));
    }
  } else {
    const int G2 = d.G >> 1;
    for (int b2 = blockIdx.x * blockDim.x + threadIdx.x; b2 < G2; b2 += gridDim.x * blockDim.x) {
      const float2 rv = finish_pair<STRETCH>(d, c, b2, M2, Mf2, F2, tA, inv_a, tf, acc, m_over,
                                             n_over, q2);
      if (d.tc)
        store_bf16_pair(d.rho_h + (size_t)c * d.G, d.rho_l + (size_t)c * d.G, b2, rv.x, rv.y);
      else
        reinterpret_cast<float2 *>(d.rho + (size_t)c * d.G)[b2] = rv;
    }
  }
  acc += ((u128)m_over << d.t_shift) - (u128)n_over * tA;
  q2 = block_sum_f<kThreads>(q2, smf);
  u128 r = block_sum_u128<kThreads>(acc, sm);
  if (threadIdx.x == 0) {
    unsigned long long *p = d.tau_part + ((size_t)c * d.nb_red + blockIdx.x) * 2;
    p[0] = (unsigned long long)r;
    p[1] = (unsigned long long)(r >> 64);
    d.conc_part[(size_t)c * d.nb_red + blockIdx.x] = q2;
  }
  if (!arrive_last(d.ctr + (size_t)c * C_COUNT + C_FINISH, &flag)) return;
  u128 v = 0;
  q2 = 0.f;
#pragma unroll 4
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    const unsigned long long *p = d.tau_part + ((size_t)c * d.nb_red + i) * 2;
    v += ((u128)p[1] << 64) | p[0];
    q2 += d.conc_part[(size_t)c * d.nb_red + i];
  }
  v = block_sum_u128<kThreads>(v, sm);
  q2 = block_sum_f<kThreads>(q2, smf);
  if (threadIdx.x == 0) {
    const double tau = ldexp(u128_to_double(v), -d.t_shift) / d.mov_area_q;
    const double s1 = (d.mov_area_q + d.fill_area_q) / d.abin_q;
    if (mode != FIN_EVAL) cs->n_eff = q2 > 0.f ? s1 * s1 / (double)q2 : 0.0;
    if (mode == FIN_ITER) {
      cs->tau = tau;
      if (tau <= (double)d.prm.tau_stop) cs->converged = cs->stopped = 1;
    } else if (mode == FIN_RESET) {
      cs->tau = cs->tau_prev = tau;
      cs->gamma = gamma_of(d, tau);
      if (d.prm.max_iters <= 0) cs->stopped = 1;
    } else {
      d.scal[(size_t)c * S_COUNT + S_TAU] = tau;
    }
    d.ctr[(size_t)c * C_COUNT + C_FINISH] = 0u;
  }
}

// Floor of the scatter's memory work at the current positions: per movable
// cell the same loads (position and quantised size) and one 64-bit reduction
// into each bin the cell covers (the bins from an FP32 estimate of its
// corners), none of the exact rectangle arithmetic.  It adds into the map,
// which the caller clears.
__global__ void __launch_bounds__(kThreads) k_scatter_floor(Dev d, int copy0) {
  const int c = copy0 + blockIdx.y;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  unsigned long long *M = d.M + (size_t)c * d.Gm;
  const float is = 1.f / d.scale;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    const int mo = i < d.n_real ? 0 : d.G;
    const float2 v = xy[i];
    const float w = (float)d.Wq[i] * is, h = (float)d.Hq[i] * is;
    const int ix0 = min(max((int)floorf((v.x - d.fxl) * d.fibw), 0), d.nx - 1);
    const int ix1 = min(max((int)floorf((v.x + w - d.fxl) * d.fibw), 0), d.nx - 1);
    const int iy0 = min(max((int)floorf((v.y - d.fyl) * d.fibh), 0), d.ny - 1);
    const int iy1 = min(max((int)floorf((v.y + h - d.fyl) * d.fibh), 0), d.ny - 1);
    for (int ix = ix0; ix <= ix1; ++ix)
      for (int iy = iy0; iy <= iy1; ++iy) {
        const int b = mo + ix * d.ny + iy;
        if (HP_IN(d.err, b, d.Gm, BS_MAP_BIN)) atomicAdd(&M[b], 1ull);
      }
  }
}

void launch_scatter_floor(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  k_scatter_floor<<<dim3(d.cell_blocks, ncopy), kThreads, 0, st>>>(d, copy0);
}

void launch_scatter_main(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st) {
  k_scatter<<<dim3(d.cell_blocks, ncopy), kThreads, 0, st>>>(d, copy0, eval);
}

void launch_scatter(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st) {
  dim3 grid(d.cell_blocks, ncopy);
  k_scatter<<<grid, kThreads, 0, st>>>(d, copy0, eval);
  if (d.Ms) {
    cudaMemsetAsync(d.Ms + (size_t)copy0 * d.G, 0, sizeof(unsigned long long) * d.G * ncopy, st);
    k_scatter_stretch<<<grid, kThreads, 0, st>>>(d, copy0, eval);
  }
}

void launch_scatter_fixed(const Dev &d, const float2 *xy, int n0, int n1,
                          unsigned long long *out, cudaStream_t st) {
  if (n1 <= n0) return;
  int blocks = (n1 - n0 + kThreads - 1) / kThreads;
  if (blocks > 4096) blocks = 4096;
  k_scatter_range<<<blocks, kThreads, 0, st>>>(d, xy, n0, n1, out);
}

void launch_density_finish(const Dev &d, int copy0, int ncopy, int mode, cudaStream_t st) {
  dim3 grid(d.bin_blocks, ncopy);
  if (d.Ms && d.bfly)
    launch_pdl(k_density_finish<true, true>, grid, dim3(kThreads), 0, st, d, copy0, mode);
  else if (d.Ms)
    launch_pdl(k_density_finish<true, false>, grid, dim3(kThreads), 0, st, d, copy0, mode);
  else if (d.bfly)
    launch_pdl(k_density_finish<false, true>, grid, dim3(kThreads), 0, st, d, copy0, mode);
  else
    launch_pdl(k_density_finish<false, false>, grid, dim3(kThreads), 0, st, d, copy0, mode);
}

}  // namespace hp
