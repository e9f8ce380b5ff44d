// Electrostatic density: exact overlap-area bin map in 64-bit fixed point and
// its conversion to bin density and overflow.
//
// The density D of Eq. 1/2 is the ePlace electrostatic density the paper
// cites.  Reading: coordinates quantised to multiples of 2^-F (x * 2^F is
// exact in FP32, rounded to the nearest integer with ties to even), movable
// map M_b = sum_i overlap(cell_i, bin_b) as int64 in units of 2^-2F,
// overflow tau = sum_b max(0, M_b - t (A_b - F_b)) / A_mov and bin density
// rho_b = (M_b + t F_b) / A_b.  Integer addition is associative, so the map
// is bit-exact and independent of the order in which cells are added.
#include "common.cuh"
#include "internal.cuh"

namespace hp {

// One thread per movable cell; each adds its integer overlap areas to the
// copy's map with 64-bit integer atomics.
__global__ void __launch_bounds__(kThreads) k_scatter(Dev d, int copy0, int eval) {
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
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
        atomicAdd(&M[(size_t)ix * d.ny + iy], (unsigned long long)(ox * oy));
      }
    }
  }
}

// Same for an arbitrary cell range (the fixed cells, once at create).
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

// Per bin: overflow excess (FP64 partial per block) and rho in FP32.
__global__ void __launch_bounds__(kThreads) k_density_finish(Dev d, int copy0, int eval) {
  __shared__ double sm[32];
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  const unsigned long long *M = d.M + (size_t)c * d.G;
  float *rho = d.rho + (size_t)c * d.G;
  double s = 0.0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.G; b += gridDim.x * blockDim.x) {
    double m = (double)(long long)M[b];
    double f = (double)d.Fmap[b];
    double ex = m - d.t * (d.abin_q - f);
    s += ex > 0.0 ? ex : 0.0;
    rho[b] = (float)((m + d.t * f) / d.abin_q);
  }
  double r = block_sum<kThreads>(s, sm);
  if (threadIdx.x == 0) d.part[((size_t)c * S_COUNT + S_TAU) * d.nb_red + blockIdx.x] = r;
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

void launch_density_finish(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st) {
  dim3 grid(d.bin_blocks, ncopy);
  k_density_finish<<<grid, kThreads, 0, st>>>(d, copy0, eval);
}

}  // namespace hp
