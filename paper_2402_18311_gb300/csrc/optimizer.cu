// Per-cell gradient assembly, preconditioning, the Nesterov/Lipschitz update
// and the per-copy scalar schedule (Eq. 2 minimised by Nesterov's method, as
// in the ePlace/DREAMPlace placers the paper runs in Algorithm 1 line 3).
//
// Iteration k at reference point v_k (this library's reading; the paper
// cites the method without restating it):
//   gamma_k = gamma_base w_bin 10^((20/9) tau_{k-1} - 11/9)
//   g_k = (gWL + lambda gD) / max(1, pins_i + lambda area_i)
//   alpha_k = alpha0 w_bin / rms(g_0) at k = 0, else |v_k - v_{k-1}| / |g_k - g_{k-1}|
//   u_{k+1} = clamp(v_k - alpha_k g_k)
//   a_{k+1} = (1 + sqrt(4 a_k^2 + 1)) / 2
//   v_{k+1} = clamp(u_{k+1} + (a_k - 1)/a_{k+1} (u_{k+1} - u_k))
//   lambda_0 = eta |gWL|_1 / |gD|_1;  lambda_{k+1} = lambda_k clamp(mu^(1 - dHPWL/dref))
// Per-cell work is FP32; norms and scalars are FP64, reduced in a fixed
// order so that every run of the same input gives the same bits.
#include <math.h>

#include "common.cuh"
#include "internal.cuh"

namespace hp {

__device__ __forceinline__ double *part_ptr(const Dev &d, int c, int slot) {
  return d.part + ((size_t)c * S_COUNT + slot) * d.nb_red;
}

// Gradient of the wirelength (sum of the cell's pin gradients) and of the
// density (field gather -sum_b a_ib E_b) for every movable cell.  For k >= 1
// (lambda known) the preconditioned gradient and the step-size norms are
// formed here too.
__global__ void __launch_bounds__(kThreads) k_cell_grad(Dev d, int copy0, int eval) {
  __shared__ double sm[32];
  const int c = copy0 + blockIdx.y;
  const CopyState &cs = d.cs[c];
  if (!eval && cs.stopped) return;
  const int k = cs.k;
  const bool full = !eval && k >= 1;
  const float lam = (float)cs.lam;
  const int par = cs.parity;
  const size_t cn = (size_t)c * d.n_cells, cm = (size_t)c * d.n_mov;
  const float *x = d.x + cn, *y = d.y + cn;
  const float2 *pg = d.pin_grad + (size_t)c * d.n_pins;
  const float *ex = d.E + (size_t)c * 3 * d.G, *ey = ex + d.G;
  double n1 = 0, d1 = 0, dg2 = 0, dv2 = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    float sx = 0.f, sy = 0.f;
    for (int q = d.cell_pin_ptr[i]; q < d.cell_pin_ptr[i + 1]; ++q) {
      float2 g = pg[d.cell_pins[q]];
      sx += g.x;
      sy += g.y;
    }
    const float xi = x[i], yi = y[i];
    QRect r = qrect(xi, yi, d.Wq[i], d.Hq[i], d.scale, d.XL, d.YL, d.BW, d.BH, d.nx, d.ny);
    float dx = 0.f, dy = 0.f;
    for (int ix = r.ix0; ix <= r.ix1; ++ix) {
      long long ox = overlap1(r.X, r.W, d.XL + (long long)ix * d.BW, d.BW);
      if (ox == 0) continue;
      for (int iy = r.iy0; iy <= r.iy1; ++iy) {
        long long oy = overlap1(r.Y, r.H, d.YL + (long long)iy * d.BH, d.BH);
        if (oy == 0) continue;
        float a = (float)(ox * oy) * d.inv_area_q;
        size_t b = (size_t)ix * d.ny + iy;
        dx -= a * ex[b];
        dy -= a * ey[b];
      }
    }
    d.gwx[cm + i] = sx; d.gwy[cm + i] = sy;
    d.gdx[cm + i] = dx; d.gdy[cm + i] = dy;
    n1 += fabs((double)sx) + fabs((double)sy);
    d1 += fabs((double)dx) + fabs((double)dy);
    if (full) {
      float P = fmaxf(1.f, d.npins[i] + lam * d.area[i]);
      float gx = (sx + lam * dx) / P, gy = (sy + lam * dy) / P;
      d.gx[par][cm + i] = gx;
      d.gy[par][cm + i] = gy;
      double ax = (double)gx - (double)d.gx[par ^ 1][cm + i];
      double ay = (double)gy - (double)d.gy[par ^ 1][cm + i];
      dg2 += ax * ax + ay * ay;
      double bx = (double)xi - (double)d.vpx[cm + i];
      double by = (double)yi - (double)d.vpy[cm + i];
      dv2 += bx * bx + by * by;
    }
  }
  double r0 = block_sum<kThreads>(n1, sm);
  double r1 = block_sum<kThreads>(d1, sm);
  double r2 = block_sum<kThreads>(dg2, sm);
  double r3 = block_sum<kThreads>(dv2, sm);
  if (threadIdx.x == 0) {
    part_ptr(d, c, S_GW1)[blockIdx.x] = r0;
    part_ptr(d, c, S_GD1)[blockIdx.x] = r1;
    part_ptr(d, c, S_DG2)[blockIdx.x] = r2;
    part_ptr(d, c, S_DV2)[blockIdx.x] = r3;
  }
}

// k == 0 only: preconditioned gradient once lambda_0 is known, and |g|^2.
__global__ void __launch_bounds__(kThreads) k_precond0(Dev d, int copy0) {
  __shared__ double sm[32];
  const int c = copy0 + blockIdx.y;
  const CopyState &cs = d.cs[c];
  if (cs.stopped || cs.k != 0) return;
  const float lam = (float)cs.lam;
  const int par = cs.parity;
  const size_t cm = (size_t)c * d.n_mov;
  double g2 = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    float P = fmaxf(1.f, d.npins[i] + lam * d.area[i]);
    float gx = (d.gwx[cm + i] + lam * d.gdx[cm + i]) / P;
    float gy = (d.gwy[cm + i] + lam * d.gdy[cm + i]) / P;
    d.gx[par][cm + i] = gx;
    d.gy[par][cm + i] = gy;
    g2 += (double)gx * gx + (double)gy * gy;
  }
  double r = block_sum<kThreads>(g2, sm);
  if (threadIdx.x == 0) part_ptr(d, c, S_G2)[blockIdx.x] = r;
}

// Nesterov step with clamping into the die.
__global__ void __launch_bounds__(kThreads) k_update(Dev d, int copy0) {
  const int c = copy0 + blockIdx.y;
  const CopyState &cs = d.cs[c];
  if (cs.stopped) return;
  const float alpha = (float)cs.alpha, coef = (float)cs.coef;
  const int par = cs.parity;
  const size_t cn = (size_t)c * d.n_cells, cm = (size_t)c * d.n_mov;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    const float xh = d.fxh - d.w[i], yh = d.fyh - d.h[i];
    const float vx = d.x[cn + i], vy = d.y[cn + i];
    const float ux = d.ux[cm + i], uy = d.uy[cm + i];
    float nux = fmaxf(d.fxl, fminf(vx - alpha * d.gx[par][cm + i], xh));
    float nuy = fmaxf(d.fyl, fminf(vy - alpha * d.gy[par][cm + i], yh));
    float nvx = fmaxf(d.fxl, fminf(nux + coef * (nux - ux), xh));
    float nvy = fmaxf(d.fyl, fminf(nuy + coef * (nuy - uy), yh));
    d.vpx[cm + i] = vx; d.vpy[cm + i] = vy;
    d.ux[cm + i] = nux; d.uy[cm + i] = nuy;
    d.x[cn + i] = nvx; d.y[cn + i] = nvy;
  }
}

// Optimiser reset: clamp the movable positions into the die, u = v, and
// initial scalars.
__global__ void __launch_bounds__(kThreads) k_reset(Dev d, int copy0) {
  const int c = copy0 + blockIdx.y;
  const size_t cn = (size_t)c * d.n_cells, cm = (size_t)c * d.n_mov;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    float vx = fmaxf(d.fxl, fminf(d.x[cn + i], d.fxh - d.w[i]));
    float vy = fmaxf(d.fyl, fminf(d.y[cn + i], d.fyh - d.h[i]));
    d.x[cn + i] = vx; d.y[cn + i] = vy;
    d.ux[cm + i] = vx; d.uy[cm + i] = vy;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CopyState s = {};
    s.a = 1.0;
    d.cs[c] = s;
  }
}

// Deterministic sum of one slot's block partials: strided per-thread sums,
// then a fixed tree.
__device__ double reduce_slot(const Dev &d, int c, int slot, int nvals, double *sm) {
  const double *p = part_ptr(d, c, slot);
  double v = 0.0;
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) v += p[i];
  double r = block_sum<kRedThreads>(v, sm);
  __syncthreads();
  if (threadIdx.x == 0) sm[32] = r;
  __syncthreads();
  r = sm[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kRedThreads) k_scalars(Dev d, int phase, int copy0) {
  __shared__ double sm[40];
  const int c = copy0 + blockIdx.x;
  CopyState *cs = d.cs + c;
  const place_params &P = d.prm;
  if (phase == PH_TAU_RESET) {
    double s = reduce_slot(d, c, S_TAU, d.bin_blocks, sm);
    if (threadIdx.x == 0) cs->tau = cs->tau_prev = s / d.mov_area_q;
    return;
  }
  if (cs->stopped) return;
  switch (phase) {
    case PH_BEGIN:
      if (threadIdx.x == 0) {
        if (cs->k >= P.max_iters) {
          cs->stopped = 1;
        } else if (P.constant_gamma > 0.f) {
          cs->gamma = (double)P.constant_gamma;
        } else {
          cs->gamma = (double)P.gamma_base * d.w_bin *
                      pow(10.0, (20.0 / 9.0) * cs->tau_prev - 11.0 / 9.0);
        }
      }
      break;
    case PH_TAU: {
      double s = reduce_slot(d, c, S_TAU, d.bin_blocks, sm);
      if (threadIdx.x == 0) {
        double tau = s / d.mov_area_q;
        cs->tau = tau;
        if (tau <= (double)P.tau_stop) cs->converged = cs->stopped = 1;
      }
      break;
    }
    case PH_MID: {
      double hp = reduce_slot(d, c, S_HPWL, d.wa_blocks_total, sm);
      double wl = reduce_slot(d, c, S_WL, d.wa_blocks_total, sm);
      double n1 = 0, d1 = 0;
      const bool first = cs->k == 0;
      if (first) {
        n1 = reduce_slot(d, c, S_GW1, d.cell_blocks, sm);
        d1 = reduce_slot(d, c, S_GD1, d.cell_blocks, sm);
      }
      if (threadIdx.x == 0) {
        cs->hpwl = hp;
        cs->wl = wl;
        if (first) cs->lam = d1 > 0 ? (double)P.lambda_eta * n1 / d1 : (double)P.lambda_eta;
      }
      break;
    }
    case PH_ALPHA: {
      const bool first = cs->k == 0;
      double g2 = 0, dv2 = 0, dg2 = 0;
      if (first) {
        g2 = reduce_slot(d, c, S_G2, d.cell_blocks, sm);
      } else {
        dv2 = reduce_slot(d, c, S_DV2, d.cell_blocks, sm);
        dg2 = reduce_slot(d, c, S_DG2, d.cell_blocks, sm);
      }
      if (threadIdx.x == 0) {
        double alpha;
        if (first) {
          double rms = sqrt(g2 / (2.0 * d.n_mov));
          alpha = rms > 0 ? (double)P.alpha0 * d.w_bin / rms : 0.0;
        } else {
          alpha = dg2 > 0 ? sqrt(dv2) / sqrt(dg2) : cs->alpha;
        }
        cs->alpha = alpha;
        cs->a_next = (1.0 + sqrt(4.0 * cs->a * cs->a + 1.0)) / 2.0;
        cs->coef = (cs->a - 1.0) / cs->a_next;
        if (!first) {
          double mu = pow((double)P.mu_base, 1.0 - (cs->hpwl - cs->hpwl_prev) / d.dref);
          mu = fmin(fmax(mu, (double)P.mu_lo), (double)P.mu_hi);
          cs->lam *= mu;
        }
        cs->hpwl_prev = cs->hpwl;
        cs->tau_prev = cs->tau;
      }
      break;
    }
    case PH_END:
      if (threadIdx.x == 0) {
        cs->k += 1;
        cs->a = cs->a_next;
        cs->parity ^= 1;
        if (cs->k >= P.max_iters) cs->stopped = 1;
      }
      break;
  }
}

// Reduce one slot for evaluation calls: d.scal[c * S_COUNT + slot].
__global__ void __launch_bounds__(kRedThreads) k_reduce_slot(Dev d, int slot, int nvals,
                                                             int copy0) {
  __shared__ double sm[40];
  const int c = copy0 + blockIdx.x;
  double s = reduce_slot(d, c, slot, nvals, sm);
  if (threadIdx.x == 0) d.scal[(size_t)c * S_COUNT + slot] = s;
}

void launch_cell_grad(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st) {
  k_cell_grad<<<dim3(d.cell_blocks, ncopy), kThreads, 0, st>>>(d, copy0, eval);
}
void launch_precond0(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  k_precond0<<<dim3(d.cell_blocks, ncopy), kThreads, 0, st>>>(d, copy0);
}
void launch_update(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  k_update<<<dim3(d.cell_blocks, ncopy), kThreads, 0, st>>>(d, copy0);
}
void launch_reset(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  k_reset<<<dim3(d.cell_blocks, ncopy), kThreads, 0, st>>>(d, copy0);
}
void launch_iteration_scalars(const Dev &d, int phase, int copy0, int ncopy, cudaStream_t st) {
  k_scalars<<<ncopy, kRedThreads, 0, st>>>(d, phase, copy0);
}
void launch_reduce_slot(const Dev &d, int slot, int nvals, int copy0, int ncopy,
                        cudaStream_t st) {
  k_reduce_slot<<<ncopy, kRedThreads, 0, st>>>(d, slot, nvals, copy0);
}

}  // namespace hp
