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

// Cells are processed grid-stride; each block first aggregates its overlap
// areas per bin in a shared-memory hash table (bounded linear probing) and
// flushes the table with one 64-bit atomic per distinct bin.  Contributions
// that find no slot go straight to global memory.  When many cells share
// few bins (the centred start of a placement) this removes almost all
// contention on the global map.
__global__ void __launch_bounds__(kThreads) k_scatter(Dev d, int copy0, int eval) {
  __shared__ int keys[kHash];
  __shared__ unsigned long long vals[kHash];
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  for (int i = threadIdx.x; i < kHash; i += blockDim.x) {
    keys[i] = -1;
    vals[i] = 0ull;
  }
  __syncthreads();
  const float *x = d.x + (size_t)c * d.n_cells;
  const float *y = d.y + (size_t)c * d.n_cells;
  unsigned long long *M = d.M + (size_t)c * d.G;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    QRect r = qrect(x[i], y[i], d.Wq[i], d.Hq[i], d.scale, d.XL, d.YL, d.BW, d.BH, d.nx, d.ny);
    for (int ix = r.ix0; ix <= r.ix1; ++ix) {
      long long ox = overlap1(r.X, r.W, d.XL + (long long)ix * d.BW, d.BW);
      if (ox == 0) continue;
      for (int iy = r.iy0; iy <= r.iy1; ++iy) {
        long long oy = overlap1(r.Y, r.H, d.YL + (long long)iy * d.BH, d.BH);
        if (oy == 0) continue;
        const int b = ix * d.ny + iy;
        const unsigned long long a = (unsigned long long)(ox * oy);
        unsigned int hsh = ((unsigned int)b * 2654435761u) >> (32 - 11);
        bool done = false;
#pragma unroll 1
        for (int probe = 0; probe < 2; ++probe) {
          int k = keys[hsh];  // plain read first: no atomic when the bin is already there
          if (k == -1) k = atomicCAS(&keys[hsh], -1, b);
          if (k == -1 || k == b) {
            atomicAdd(&vals[hsh], a);
            done = true;
            break;
          }
          hsh = (hsh + 1) & (kHash - 1);
        }
        if (!done) atomicAdd(&M[b], a);
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
    k_scatter_range(Dev d, const float *x, const float *y, int n0, int n1,
                    unsigned long long *out) {
  for (int i = n0 + blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) {
    QRect r = qrect(x[i], y[i], d.Wq[i], d.Hq[i], d.scale, d.XL, d.YL, d.BW, d.BH, d.nx, d.ny);
    for (int ix = r.ix0; ix <= r.ix1; ++ix) {
      long long ox = overlap1(r.X, r.W, d.XL + (long long)ix * d.BW, d.BW);
      if (ox == 0) continue;
      for (int iy = r.iy0; iy <= r.iy1; ++iy) {
        long long oy = overlap1(r.Y, r.H, d.YL + (long long)iy * d.BH, d.BH);
        if (oy == 0) continue;
        atomicAdd(&out[(size_t)ix * d.ny + iy], (unsigned long long)(ox * oy));
      }
    }
  }
}

// Per bin: exact overflow excess and rho in FP32; the last block of each copy
// reduces the excess and, by mode, records the overflow as the iteration's
// tau (with the stop test), as an evaluation result, or as the reset value
// tau_{-1} that sets the first gamma.
__global__ void __launch_bounds__(kThreads) k_density_finish(Dev d, int copy0, int mode) {
  __shared__ u128 sm[32];
  __shared__ int flag;
  const int c = copy0 + blockIdx.y;
  CopyState *cs = d.cs + c;
  if (mode == FIN_ITER && cs->stopped) return;
  const unsigned long long *M = d.M + (size_t)c * d.G;
  float *rho = d.rho + (size_t)c * d.G;
  const long long abin = d.BW * d.BH;
  const float inv_a = (float)(1.0 / d.abin_q);
  const float tf = (float)d.t;
  u128 acc = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.G; b += gridDim.x * blockDim.x) {
    const long long m = (long long)M[b];
    const long long f = d.Fmap[b];
    // excess * 2^s = m 2^s - t_mant (A - F): exact in 128 bits
    const __int128 e = ((__int128)m << d.t_shift) - (__int128)d.t_mant * (__int128)(abin - f);
    if (e > 0) acc += (u128)e;
    const float rv = (float)m * inv_a + tf * ((float)f * inv_a);
    if (d.tc) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(rv);
      d.rho_h[(size_t)c * d.G + b] = hi;
      d.rho_l[(size_t)c * d.G + b] = __float2bfloat16_rn(rv - __bfloat162float(hi));
    } else {
      rho[b] = rv;
    }
  }
  u128 r = block_sum_u128<kThreads>(acc, sm);
  if (threadIdx.x == 0) {
    unsigned long long *p = d.tau_part + ((size_t)c * d.nb_red + blockIdx.x) * 2;
    p[0] = (unsigned long long)r;
    p[1] = (unsigned long long)(r >> 64);
  }
  if (!arrive_last(d.ctr + (size_t)c * C_COUNT + C_FINISH, &flag)) return;
  u128 v = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    const unsigned long long *p = d.tau_part + ((size_t)c * d.nb_red + i) * 2;
    v += ((u128)p[1] << 64) | p[0];
  }
  v = block_sum_u128<kThreads>(v, sm);
  if (threadIdx.x == 0) {
    const double tau = ldexp(u128_to_double(v), -d.t_shift) / d.mov_area_q;
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

void launch_scatter(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st) {
  dim3 grid(d.cell_blocks, ncopy);
  k_scatter<<<grid, kThreads, 0, st>>>(d, copy0, eval);
}

void launch_scatter_fixed(const Dev &d, const float *x, const float *y, int n0, int n1,
                          unsigned long long *out, cudaStream_t st) {
  if (n1 <= n0) return;
  int blocks = (n1 - n0 + kThreads - 1) / kThreads;
  if (blocks > 4096) blocks = 4096;
  k_scatter_range<<<blocks, kThreads, 0, st>>>(d, x, y, n0, n1, out);
}

void launch_density_finish(const Dev &d, int copy0, int ncopy, int mode, cudaStream_t st) {
  dim3 grid(d.bin_blocks, ncopy);
  k_density_finish<<<grid, kThreads, 0, st>>>(d, copy0, mode);
}

}  // namespace hp
