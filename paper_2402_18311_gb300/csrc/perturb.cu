// Shuffle and Shuffle (all) perturbations (the perturbation step of
// Algorithm 1; Section 4.2: a random fraction p of the macros, or of all the
// cells, exchange their locations among themselves).  Reading used by this
// library:
//   - every cell i draws r_i, the (i+1)-th output of SplitMix64 started from
//     `seed` (Steele, Lea and Flood, OOPSLA 2014), evaluated directly from
//     its counter: state = seed + (i+1) * 0x9E3779B97F4A7C15, then the mix;
//   - the k = floor(p n + 1/2) candidates with the smallest (r_i, i) are
//     selected; candidates are the movable macros (Shuffle) or all movable
//     cells (Shuffle (all));
//   - taking the selected cells in key order t_0, t_1, ... and in index order
//     s_0 < s_1 < ..., cell t_j receives the centre of cell s_j, clamped into
//     the die.  New corners are computed in FP64 and rounded once.
// Selection and permutation are integer work and bit-exact; they run as a
// bitonic sort over (key, index) pairs.
#include "common.cuh"
#include "internal.cuh"

namespace hp {

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr unsigned int kNotCand = 0x80000000u;

__global__ void k_keys(Dev d, int op, unsigned long long seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.sort_n; i += gridDim.x * blockDim.x) {
    bool cand = i < d.n_real && (op == PLACE_SHUFFLE_ALL || d.is_macro[i]);
    if (cand) {
      d.sort_key[i] = splitmix64_at(seed, (unsigned long long)i);
      d.sort_idx[i] = (unsigned int)i;
    } else {
      d.sort_key[i] = ~0ull;
      d.sort_idx[i] = kNotCand | (unsigned int)(i & 0x7fffffff);
    }
  }
}

// One compare-exchange pass of a bitonic sort on (key, idx) pairs, ascending.
__global__ void k_bitonic(unsigned long long *key, unsigned int *idx, int n, int j, int k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int p = t ^ j;
    if (p <= t) continue;
    unsigned long long ka = key[t], kb = key[p];
    unsigned int ia = idx[t], ib = idx[p];
    bool a_gt_b = (ka > kb) || (ka == kb && ia > ib);
    bool up = (t & k) == 0;
    if (a_gt_b == up) {
      key[t] = kb; key[p] = ka;
      idx[t] = ib; idx[p] = ia;
    }
  }
}

// Index-order copy of the k selected cells (keys = index, padding = max).
__global__ void k_sel_init(Dev d, int k, int n2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    unsigned int v = i < k ? d.sort_idx[i] : 0xffffffffu;
    d.sel_idx[i] = v;
  }
}

__global__ void k_bitonic_u32(unsigned int *v, int n, int j, int k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int p = t ^ j;
    if (p <= t) continue;
    unsigned int a = v[t], b = v[p];
    bool up = (t & k) == 0;
    if ((a > b) == up) {
      v[t] = b;
      v[p] = a;
    }
  }
}

__global__ void k_shuffle_compute(Dev d, int copy, int k) {
  const float2 *xy = d.xy + (size_t)copy * d.n_cells;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
    int r = (int)d.sort_idx[j];  // receiver (key order)
    int s = (int)d.sel_idx[j];   // donor (index order)
    HP_FIX(d.err, r, d.n_real, BS_PERM);
    HP_FIX(d.err, s, d.n_real, BS_PERM);
    const float2 ps = xy[s];
    double cx = (double)ps.x + 0.5 * (double)d.w[s];
    double cy = (double)ps.y + 0.5 * (double)d.h[s];
    double nx = cx - 0.5 * (double)d.w[r];
    double ny = cy - 0.5 * (double)d.h[r];
    nx = fmax(d.die_xl, fmin(nx, d.die_xh - (double)d.w[r]));
    ny = fmax(d.die_yl, fmin(ny, d.die_yh - (double)d.h[r]));
    d.px_tmp[j] = (float)nx;
    d.py_tmp[j] = (float)ny;
  }
}

__global__ void k_shuffle_apply(Dev d, int copy, int k) {
  float2 *xy = d.xy + (size_t)copy * d.n_cells;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
    const int r = (int)d.sort_idx[j];
    if (!HP_IN(d.err, r, d.n_real, BS_PERM)) continue;
    xy[r] = make_float2(d.px_tmp[j], d.py_tmp[j]);
  }
}

static int grid_for(int n) {
  int b = (n + kThreads - 1) / kThreads;
  return b < 1 ? 1 : (b > 8192 ? 8192 : b);
}

// Returns the number of moved cells (>= 0); candidates counted on the host.
int launch_shuffle(const Dev &d, int copy, int op, float p, uint64_t seed, cudaStream_t st) {
  const int n = d.sort_n;
  k_keys<<<grid_for(n), kThreads, 0, st>>>(d, op, (unsigned long long)seed);
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1)
      k_bitonic<<<grid_for(n / 2 + 1), kThreads, 0, st>>>(d.sort_key, d.sort_idx, n, j, k);
  return 0;
}

// Second half: given the candidate count, select k and move the cells.
void launch_shuffle_finish(const Dev &d, int copy, int kcount, cudaStream_t st) {
  if (kcount <= 0) return;
  int n2 = 1;
  while (n2 < kcount) n2 <<= 1;
  if (n2 < 2) n2 = 2;
  k_sel_init<<<grid_for(n2), kThreads, 0, st>>>(d, kcount, n2);
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1)
      k_bitonic_u32<<<grid_for(n2 / 2 + 1), kThreads, 0, st>>>(d.sel_idx, n2, j, k);
  k_shuffle_compute<<<grid_for(kcount), kThreads, 0, st>>>(d, copy, kcount);
  k_shuffle_apply<<<grid_for(kcount), kThreads, 0, st>>>(d, copy, kcount);
}

}  // namespace hp
