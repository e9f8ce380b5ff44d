// WireMask perturbation (the perturbation step of Algorithm 1; Section 4.2):
// every movable macro, one after another, moves to the grid position where
// the HPWL grows least.  Reading used by this library:
//   - macros: the movable cells flagged is_macro, by decreasing area (ties
//     by index);
//   - candidates: the macro's lower-left corner on a bin corner,
//     X_i = fl32(xl + i (xh - xl)/nx), inside the die (X_i + w <= xh);
//   - wire mask: the weighted HPWL (Eq. 1) of the macro's nets with the
//     macro at the candidate and every other pin where it is (macros moved
//     earlier in the pass at their new places).  For one net, with the
//     other pins' extent [o-, o+] and the macro's pin offsets [d-, d+], the
//     x part is max(o+, X + d+) - min(o-, X + d-).  The mask is separable,
//     Fx(X_i) + Fy(Y_j), each axis summed over the macro's nets in netlist
//     order;
//   - obstacles: every fixed cell and the macros moved before this one;
//     overlap of positive area blocks a candidate (touching is allowed);
//   - choice: the smallest (Fx + Fy, |X - x| + |Y - y|, j, i) among the
//     free candidates, (x, y) the macro's position before it moves; with
//     none free the macro stays.
// Every value that decides a comparison is FP64 from a fixed sequence of
// correctly rounded operations (explicit _rn intrinsics, so no contraction
// into fused multiply-adds), so the result is bit-exact and
// independent of the launch shape.  Per macro:
//   - one warp per net computes the net's extents;
//   - one thread per grid line sums a mask axis;
//   - each block turns every obstacle into the exact range of candidate
//     columns and rows it blocks (binary searches); each candidate then
//     tests integer ranges and takes part in a block argmin;
//   - a last kernel reduces the blocks' winners and moves the macro.
// Copies run side by side (blockIdx.y).
#include <cmath>

#include "common.cuh"
#include "internal.cuh"

namespace hp {

namespace {

constexpr int kWmThreads = 256;

__device__ __forceinline__ double wm_step(double lo, double hi, int n) {
  return __ddiv_rn(__dsub_rn(hi, lo), (double)n);
}
// Candidate corner i: fl32(lo + i b) with b = (hi - lo) / n.
__device__ __forceinline__ double wm_corner_b(double lo, double b, int i) {
  return (double)__double2float_rn(__dadd_rn(lo, __dmul_rn((double)i, b)));
}
__device__ __forceinline__ double wm_corner(double lo, double hi, int n, int i) {
  return wm_corner_b(lo, wm_step(lo, hi, n), i);
}

// First k in [0, n] at which a predicate that is false and then true over
// [0, n) holds (n when it never does).
template <typename P>
__device__ __forceinline__ int first_true(int n, P pred) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (pred(mid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// The corners i whose macro rectangle [X_i, X_i + w) overlaps [o0, o1) with
// positive length: X_i < o1 and o0 < X_i + w.  The corners are
// nondecreasing in i (rounding is monotone), so the first test holds for i
// below some bound and the second from some bound on.  Two binary searches
// over the same FP64 expressions give the range [i0, i1] exactly.
__device__ __forceinline__ int2 blocked_range(double lo, double b, int n, double w, double o0,
                                              double o1) {
  const int i0 = first_true(n, [&](int i) { return o0 < __dadd_rn(wm_corner_b(lo, b, i), w); });
  const int i1 = first_true(n, [&](int i) { return !(wm_corner_b(lo, b, i) < o1); }) - 1;
  return make_int2(i0, i1);
}

struct Best {
  double obj, dist;
  int idx;  // flat candidate index j * nx + i; -1: none
};

__device__ __forceinline__ bool better(const Best &a, const Best &b) {
  if (a.idx < 0) return false;
  if (b.idx < 0) return true;
  if (a.obj != b.obj) return a.obj < b.obj;
  if (a.dist != b.dist) return a.dist < b.dist;
  return a.idx < b.idx;
}

__device__ __forceinline__ Best shfl_best(const Best &v, int o) {
  Best r;
  r.obj = __shfl_xor_sync(0xffffffffu, v.obj, o);
  r.dist = __shfl_xor_sync(0xffffffffu, v.dist, o);
  r.idx = __shfl_xor_sync(0xffffffffu, v.idx, o);
  return r;
}

// Block-wide argmin (every thread of the block calls it); result in thread 0.
__device__ Best block_best(Best v) {
  __shared__ double s_obj[kWmThreads / 32], s_dist[kWmThreads / 32];
  __shared__ int s_idx[kWmThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const Best w = shfl_best(v, o);
    if (better(w, v)) v = w;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    s_obj[threadIdx.x >> 5] = v.obj;
    s_dist[threadIdx.x >> 5] = v.dist;
    s_idx[threadIdx.x >> 5] = v.idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kWmThreads / 32; ++k) {
      const Best w{s_obj[k], s_dist[k], s_idx[k]};
      if (better(w, v)) v = w;
    }
  }
  return v;
}

// Extents of every net of macro t: one warp per net.  box[8] =
// {o-x, o+x, o-y, o+y, d-x, d+x, d-y, d+y}: other pins' coordinates and the
// macro's own pin offsets (+-inf when empty).
__global__ void __launch_bounds__(kWmThreads) k_wm_nets(Dev d, WmDev w, int t, int copy0) {
  const int c = copy0 + blockIdx.y;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  const int m = w.order[t];
  const int nn = w.mptr[t + 1] - w.mptr[t];
  const int s = blockIdx.x * (kWmThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= nn) return;  // the whole warp leaves together
  if (!HP_IN(d.err, s, w.max_nets, BS_WM_NET)) return;
  int e = w.mnet[w.mptr[t] + s];
  HP_FIX(d.err, e, d.n_nets, BS_WM_NET);
  double v[8] = {INFINITY, -INFINITY, INFINITY, -INFINITY,
                 INFINITY, -INFINITY, INFINITY, -INFINITY};
  for (int j = d.net_ptr[e] + lane; j < d.net_ptr[e + 1]; j += 32) {
    if (!HP_IN(d.err, j, d.n_pins, BS_WM_NET)) break;
    int cj = d.pin_cell[j];
    HP_FIX(d.err, cj, d.n_cells, BS_WM_CELL);
    const float2 o = d.pin_off[j];
    if (cj == m) {
      v[4] = fmin(v[4], (double)o.x); v[5] = fmax(v[5], (double)o.x);
      v[6] = fmin(v[6], (double)o.y); v[7] = fmax(v[7], (double)o.y);
    } else {
      const float2 p = xy[cj];
      const double px = __dadd_rn((double)p.x, (double)o.x);
      const double py = __dadd_rn((double)p.y, (double)o.y);
      v[0] = fmin(v[0], px); v[1] = fmax(v[1], px);
      v[2] = fmin(v[2], py); v[3] = fmax(v[3], py);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      v[k] = fmin(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
      v[k + 1] = fmax(v[k + 1], __shfl_xor_sync(0xffffffffu, v[k + 1], o));
    }
  }
  if (lane == 0) {
    double *b = w.box + ((size_t)blockIdx.y * w.max_nets + s) * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = v[k];
  }
}

// The two axes of macro t's wire mask: thread q < nx sums Fx(X_q), the
// next ny threads Fy(Y_q), over the macro's nets in order.
__global__ void __launch_bounds__(kWmThreads) k_wm_profile(Dev d, WmDev w, int t) {
  const int q = blockIdx.x * kWmThreads + threadIdx.x;
  if (q >= d.nx + d.ny) return;
  const bool isx = q < d.nx;
  const int i = isx ? q : q - d.nx;
  const double X = isx ? wm_corner(d.die_xl, d.die_xh, d.nx, i) : wm_corner(d.die_yl, d.die_yh, d.ny, i);
  const int a = isx ? 0 : 2;
  const int nn = w.mptr[t + 1] - w.mptr[t];
  const double *box = w.box + (size_t)blockIdx.y * w.max_nets * 8;
  double acc = 0.0;
  for (int s = 0; s < nn; ++s) {
    const double *b = box + (size_t)s * 8;
    const double hi = fmax(b[a + 1], __dadd_rn(X, b[a + 5]));
    const double lo = fmin(b[a], __dadd_rn(X, b[a + 4]));
    const double wn = d.net_w ? (double)d.net_w[w.mnet[w.mptr[t] + s]] : 1.0;
    acc = __dadd_rn(acc, __dmul_rn(wn, __dsub_rn(hi, lo)));
  }
  if (isx) w.fx[(size_t)blockIdx.y * d.nx + i] = acc;
  else w.fy[(size_t)blockIdx.y * d.ny + i] = acc;
}

// One thread per candidate: inside the die, free of obstacles, key; the
// block's best goes to its partial slot.  Each obstacle becomes the range of
// candidate columns and rows it blocks (blocked_range, one thread per
// obstacle, staged in shared memory), so a candidate's test is integer
// compares; with up to one block's worth of obstacles the ranges are
// formed once per block.
__global__ void __launch_bounds__(kWmThreads) k_wm_select(Dev d, WmDev w, int t, int copy0) {
  __shared__ int4 so[kWmThreads];  // blocked columns [x, y], rows [z, w]
  const int c = copy0 + blockIdx.y;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  int m = w.order[t];
  HP_FIX(d.err, m, d.n_cells, BS_WM_CELL);
  const double mw = (double)d.w[m], mh = (double)d.h[m];
  const float2 pm = xy[m];
  const int nob = w.n_fixed + t;
  const int G = d.nx * d.ny;
  const double bx = wm_step(d.die_xl, d.die_xh, d.nx), by = wm_step(d.die_yl, d.die_yh, d.ny);
  const double *fx = w.fx + (size_t)blockIdx.y * d.nx, *fy = w.fy + (size_t)blockIdx.y * d.ny;
  auto stage = [&](int o0) {
    if (o0 + (int)threadIdx.x < nob) {
      int oc = w.obst[o0 + threadIdx.x];
      HP_FIX(d.err, oc, d.n_cells, BS_WM_CELL);
      const float2 p = xy[oc];
      const int2 rx = blocked_range(d.die_xl, bx, d.nx, mw, (double)p.x,
                                    __dadd_rn((double)p.x, (double)d.w[oc]));
      const int2 ry = blocked_range(d.die_yl, by, d.ny, mh, (double)p.y,
                                    __dadd_rn((double)p.y, (double)d.h[oc]));
      so[threadIdx.x] = make_int4(rx.x, rx.y, ry.x, ry.y);
    }
  };
  const bool once = nob <= kWmThreads;
  if (once) {
    stage(0);
    __syncthreads();
  }
  Best best{0.0, 0.0, -1};
  for (int base = blockIdx.x * kWmThreads; base < G; base += gridDim.x * kWmThreads) {
    const int q = base + threadIdx.x;
    bool ok = q < G;
    int i = 0, j = 0;
    double X = 0.0, Y = 0.0;
    if (ok) {
      j = q / d.nx;
      i = q - j * d.nx;
      X = wm_corner_b(d.die_xl, bx, i);
      Y = wm_corner_b(d.die_yl, by, j);
      ok = __dadd_rn(X, mw) <= d.die_xh && __dadd_rn(Y, mh) <= d.die_yh;
    }
    for (int o0 = 0; o0 < nob; o0 += kWmThreads) {
      if (!once) {
        __syncthreads();  // the previous chunk has been read
        stage(o0);
        __syncthreads();
      }
      const int cnt = min(kWmThreads, nob - o0);
      for (int k = 0; ok && k < cnt; ++k) {
        const int4 r = so[k];
        if (i >= r.x && i <= r.y && j >= r.z && j <= r.w) ok = false;
      }
    }
    if (ok) {
      const Best v{__dadd_rn(fx[i], fy[j]),
                   __dadd_rn(fabs(__dsub_rn(X, (double)pm.x)), fabs(__dsub_rn(Y, (double)pm.y))), q};
      if (better(v, best)) best = v;
    }
  }
  best = block_best(best);
  if (threadIdx.x == 0) {
    const size_t k = (size_t)blockIdx.y * w.nblk + blockIdx.x;
    w.bobj[k] = best.obj;
    w.bdist[k] = best.dist;
    w.bidx[k] = best.idx;
  }
}

// One block per copy: the best of the partial winners moves the macro.
__global__ void __launch_bounds__(kWmThreads) k_wm_apply(Dev d, WmDev w, int t, int copy0) {
  const int c = copy0 + blockIdx.x;
  Best best{0.0, 0.0, -1};
  for (int k = threadIdx.x; k < w.nblk; k += kWmThreads) {
    const size_t s = (size_t)blockIdx.x * w.nblk + k;
    const Best v{w.bobj[s], w.bdist[s], w.bidx[s]};
    if (better(v, best)) best = v;
  }
  best = block_best(best);
  if (threadIdx.x == 0 && best.idx >= 0 && HP_IN(d.err, best.idx, d.nx * d.ny, BS_WM_BIN)) {
    const int j = best.idx / d.nx, i = best.idx - j * d.nx;
    int m = w.order[t];
    HP_FIX(d.err, m, d.n_cells, BS_WM_CELL);
    d.xy[(size_t)c * d.n_cells + m] =
        make_float2((float)wm_corner(d.die_xl, d.die_xh, d.nx, i),
                    (float)wm_corner(d.die_yl, d.die_yh, d.ny, j));
  }
}

}  // namespace

// Two blocks per SM: each block forms the obstacle ranges once and strides
// over its candidates.
int wm_select_blocks(int G) {
  const int b = (G + kWmThreads - 1) / kWmThreads;
  return b < 1 ? 1 : (b > 304 ? 304 : b);
}

void launch_wiremask(const Dev &d, const WmDev &w, const int *mptr_host, int copy0, int ncopy,
                     cudaStream_t st) {
  for (int t = 0; t < w.n_macros; ++t) {
    const int nn = mptr_host[t + 1] - mptr_host[t];
    if (nn > 0)
      k_wm_nets<<<dim3((nn + kWmThreads / 32 - 1) / (kWmThreads / 32), ncopy), kWmThreads, 0, st>>>(
          d, w, t, copy0);
    k_wm_profile<<<dim3((d.nx + d.ny + kWmThreads - 1) / kWmThreads, ncopy), kWmThreads, 0, st>>>(
        d, w, t);
    k_wm_select<<<dim3(w.nblk, ncopy), kWmThreads, 0, st>>>(d, w, t, copy0);
    k_wm_apply<<<ncopy, kWmThreads, 0, st>>>(d, w, t, copy0);
  }
}

}  // namespace hp
