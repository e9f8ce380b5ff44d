// Per-cell gradient assembly, preconditioning, the Nesterov/Lipschitz update
// and the per-copy scalar schedule (Eq. 2 minimised by Nesterov's method, as
// in the ePlace/DREAMPlace placers that the paper runs as the
// global-placement step of Algorithm 1).
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
// Per-cell work is FP32 (GB300's FP64 rate is tiny); each thread sums its
// few cells in FP32, each block sums its threads with a compensated FP32
// tree and publishes one FP64 partial; the last block of each copy reduces the partials in a fixed order
// and advances the copy's scalars, so every run of the same input gives the
// same bits and no separate scalar kernels are launched.
#include <math.h>

#include "common.cuh"
#include "internal.cuh"

namespace hp {

__device__ __forceinline__ double *part_ptr(const Dev &d, int c, int slot) {
  return d.part + ((size_t)c * S_COUNT + slot) * d.nb_red;
}

// Fixed-order sums of NS slots' partials by a whole block; valid in thread
// 0.  Four independent accumulators per slot keep 4 * NS loads in flight
// (a single running sum would wait a full L2 round trip per partial).
template <int NT, int NS>
__device__ void sum_slots(const Dev &d, int c, const int (&slots)[NS], int n, double (&out)[NS],
                          double *sm) {
  const double *p[NS];
  double v[NS][4];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    p[s] = part_ptr(d, c, slots[s]);
    v[s][0] = v[s][1] = v[s][2] = v[s][3] = 0.0;
  }
  int i = threadIdx.x;
  for (; i + 3 * NT < n; i += 4 * NT) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[s][u] += p[s][i + u * NT];
    }
  }
  for (; i < n; i += NT) {
#pragma unroll
    for (int s = 0; s < NS; ++s) v[s][0] += p[s][i];
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) out[s] = block_sum<NT>((v[s][0] + v[s][1]) + (v[s][2] + v[s][3]), sm);
}

template <int NT>
__device__ double sum_slot(const Dev &d, int c, int slot, int n, double *sm) {
  const int slots[1] = {slot};
  double out[1];
  sum_slots<NT, 1>(d, c, slots, n, out, sm);
  return out[0];
}

// Step length, momentum and lambda schedule of iteration k (thread 0 only).
__device__ void advance_scalars(const Dev &d, CopyState *cs, bool first, double g2, double dv2,
                                double dg2) {
  const place_params &P = d.prm;
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
  cs->gamma = gamma_of(d, cs->tau);
}

// Gradient of the wirelength (the cell's packed fixed-point pin-gradient sum,
// read and cleared for the next pass) and of the density (field gather -sum_b a_ib E_b) for every movable cell.
// For k >= 1 (lambda known) the preconditioned gradient and the step-size
// norms are formed here too, and the last block advances the scalars.
// STRETCH (density stretching on): the field is gathered over the cell's
// stretched rectangle and scaled by its density scale R / 2^31.
template <bool STRETCH>
__global__ void __launch_bounds__(kThreads, 3) k_cell_grad(Dev d, int copy0, int eval) {
  __shared__ double smd[32];
  __shared__ float2 smc[32];
  __shared__ int flag;
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  CopyState *cs = d.cs + c;
  if (!eval && cs->stopped) return;
  const int k = cs->k;
  const bool full = !eval && k >= 1;
  const float lam = (float)cs->lam;
  const int par = cs->parity;
  const size_t cn = (size_t)c * d.n_cells, cm = (size_t)c * d.n_mov;
  const float2 *xy = d.xy + cn;
  unsigned long long *ga = d.gacc + cm;
  const float *ex = d.E + (size_t)c * 3 * d.G, *ey = ex + d.G;
  float n1 = 0.f, d1 = 0.f, dg2 = 0.f;
  const float2 *wh = d.wh, *pa = d.pa, *go = d.g[par ^ 1] + cm;
  // every load of the next cell is issued while this cell's field gather is
  // in flight (the gather depends on the position): two cells' loads per
  // thread in flight, at 80 registers and three blocks per SM (measured on
  // the 2.1M-cell design: the stage 0.062 -> 0.059 ms at iteration 500, the
  // iteration 0.310 -> 0.306 ms; four blocks of 64 registers with only the
  // position prefetched, or of 40 registers, were slower)
  const int stride = gridDim.x * blockDim.x;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float2 zero2 = make_float2(0.f, 0.f);
  float2 vnext = i < d.n_mov ? xy[i] : zero2, whn = i < d.n_mov ? wh[i] : zero2;
  unsigned long long gsn = i < d.n_mov ? ga[i] : 0ull;
  float2 pan = zero2, gon = zero2;
  if (full && i < d.n_mov) {
    pan = pa[i]; gon = go[i];
  }
  for (; i < d.n_mov; i += stride) {
    const unsigned long long gs = gsn;
    const float2 vi = vnext;
    const float wi = whn.x, hi = whn.y;
    const float np = pan.x, ar = pan.y, gxp = gon.x, gyp = gon.y;
    const int in = i + stride;
    if (in < d.n_mov) {
      vnext = xy[in];
      whn = wh[in];
      gsn = ga[in];
      if (full) {
        pan = pa[in]; gon = go[in];
      }
    }
    ga[i] = 0ull;
    const float2 sw = unpack_grad(d, gs);
    const float sx = sw.x, sy = sw.y;
    // density gradient: -sum_b |cell ∩ b| E_b over the bins the cell covers,
    // in FP32 with coordinates relative to the first bin's corner (exact
    // subtractions, so each overlap keeps FP32 relative precision)
    const float xi = vi.x, yi = vi.y;
    float xg = xi, yg = yi, wg = wi, hg = hi, scale_g = 1.f;
    if constexpr (STRETCH) {
      const int4 st = d.st[i];
      xg = xi - (float)st.x * d.inv_scale;
      yg = yi - (float)st.y * d.inv_scale;
      wg = (float)st.z * d.inv_scale;
      hg = (float)st.w * d.inv_scale;
      scale_g = (float)d.sR[i] * 4.656612873077393e-10f;  // 2^-31
    }
    const int ix0 = min(max((int)floorf((xg - d.fxl) * d.fibw), 0), d.nx - 1);
    const int iy0 = min(max((int)floorf((yg - d.fyl) * d.fibh), 0), d.ny - 1);
    const float rx = xg - (d.fxl + (float)ix0 * d.fbw), ry = yg - (d.fyl + (float)iy0 * d.fbh);
    const float rx1 = rx + wg, ry1 = ry + hg;
    float dx = 0.f, dy = 0.f;
    if (wg <= d.fbw && hg <= d.fbh) {
      // no larger than a bin: at most the 2 x 2 bins from (ix0, iy0), the
      // far ones loaded only where the cell reaches them
      const float ox0 = fmaxf(fminf(rx1, d.fbw) - fmaxf(rx, 0.f), 0.f);
      const float oy0 = fmaxf(fminf(ry1, d.fbh) - fmaxf(ry, 0.f), 0.f);
      const float ox1 = ix0 + 1 < d.nx ? fmaxf(rx1 - d.fbw, 0.f) : 0.f;
      const float oy1 = iy0 + 1 < d.ny ? fmaxf(ry1 - d.fbh, 0.f) : 0.f;
      const size_t b0 = (size_t)ix0 * d.ny + iy0;
      if (!HP_IN(d.err, (long long)b0 + (ox1 > 0.f ? d.ny : 0) + (oy1 > 0.f ? 1 : 0), d.G,
                 BS_FIELD_BIN))
        continue;
      const float e00x = ex[b0], e00y = ey[b0];
      const float e01x = oy1 > 0.f ? ex[b0 + 1] : 0.f, e01y = oy1 > 0.f ? ey[b0 + 1] : 0.f;
      const float e10x = ox1 > 0.f ? ex[b0 + d.ny] : 0.f, e10y = ox1 > 0.f ? ey[b0 + d.ny] : 0.f;
      const bool far = ox1 > 0.f && oy1 > 0.f;
      const float e11x = far ? ex[b0 + d.ny + 1] : 0.f, e11y = far ? ey[b0 + d.ny + 1] : 0.f;
      dx = -(ox0 * fmaf(oy0, e00x, oy1 * e01x) + ox1 * fmaf(oy0, e10x, oy1 * e11x));
      dy = -(ox0 * fmaf(oy0, e00y, oy1 * e01y) + ox1 * fmaf(oy0, e10y, oy1 * e11y));
    } else {
      for (int kx = 0, ix = ix0; ix < d.nx && (float)kx * d.fbw < rx1; ++kx, ++ix) {
        const float ox = fminf(rx1, (float)(kx + 1) * d.fbw) - fmaxf(rx, (float)kx * d.fbw);
        if (!(ox > 0.f)) continue;
        const float *exr = ex + (size_t)ix * d.ny, *eyr = ey + (size_t)ix * d.ny;
        for (int ky = 0, iy = iy0; iy < d.ny && (float)ky * d.fbh < ry1; ++ky, ++iy) {
          const float oy = fminf(ry1, (float)(ky + 1) * d.fbh) - fmaxf(ry, (float)ky * d.fbh);
          if (!(oy > 0.f)) continue;
          const float a = ox * oy;
          if (!HP_IN(d.err, (long long)ix * d.ny + iy, d.G, BS_FIELD_BIN)) continue;
          dx = fmaf(-a, exr[iy], dx);
          dy = fmaf(-a, eyr[iy], dy);
        }
      }
    }
    if constexpr (STRETCH) {
      dx *= scale_g;
      dy *= scale_g;
    }
    if (!full) {  // raw gradients are read only by k = 0 (lambda_0) and evaluations
      d.gwx[cm + i] = sx; d.gwy[cm + i] = sy;
      d.gdx[cm + i] = dx; d.gdy[cm + i] = dy;
    }
    n1 += fabsf(sx) + fabsf(sy);
    d1 += fabsf(dx) + fabsf(dy);
    if (full) {
      const float rP = 1.f / fmaxf(1.f, np + lam * ar);
      const float gx = (sx + lam * dx) * rP, gy = (sy + lam * dy) * rP;
      d.g[par][cm + i] = make_float2(gx, gy);
      const float ax = gx - gxp, ay = gy - gyp;
      dg2 += ax * ax + ay * ay;
    }
  }
  // per-thread sums in FP32 (a few cells each), compensated block sums:
  // these norms set lambda_0 and every step length
  const double r0 = block_sum_fc<kThreads>(n1, smc);
  const double r1 = block_sum_fc<kThreads>(d1, smc);
  const double r2 = block_sum_fc<kThreads>(dg2, smc);
  if (threadIdx.x == 0) {
    part_ptr(d, c, S_GW1)[blockIdx.x] = r0;
    part_ptr(d, c, S_GD1)[blockIdx.x] = r1;
    part_ptr(d, c, S_DG2)[blockIdx.x] = r2;
  }
  if (eval) return;
  if (!arrive_last(d.ctr + (size_t)c * C_COUNT + C_CELL, &flag)) return;
  const int wa_slots[2] = {S_HPWL, S_WL};
  const int cg_slots[3] = {S_GW1, S_GD1, S_DG2};
  double wa_sum[2], cg_sum[3];
  sum_slots<kThreads, 2>(d, c, wa_slots, d.wa_blocks_total, wa_sum, smd);
  sum_slots<kThreads, 3>(d, c, cg_slots, gridDim.x, cg_sum, smd);
  // |v_k - v_{k-1}|^2: the partials of the step that led here (k_update or
  // k_redo_step, one per block of their grid)
  const double s4 = k > 0 ? sum_slot<kThreads>(d, c, S_DV2, d.cell_blocks, smd) : 0.0;
  const double hp = wa_sum[0], wl = wa_sum[1];
  const double s1 = cg_sum[0], s2 = cg_sum[1], s3 = cg_sum[2];
  if (threadIdx.x == 0) {
    cs->hpwl = hp;
    cs->wl = wl;
    if (k == 0) {
      cs->lam = s2 > 0 ? (double)d.prm.lambda_eta * s1 / s2 : (double)d.prm.lambda_eta;
    } else {
      // backtracking: a step-length estimate below 0.95 times the step that
      // led here sends k_update back to redo that step with the estimate
      const double est = s3 > 0 ? sqrt(s4) / sqrt(s3) : cs->alpha;
      if (d.prm.max_backtracks > 0 && cs->n_back < d.prm.max_backtracks && est < 0.95 * cs->alpha) {
        cs->alpha = est;
        cs->n_back += 1;
        cs->n_back_total += 1;
        cs->reject = 1;
      } else {
        cs->n_back = 0;
        advance_scalars(d, cs, false, 0.0, s4, s3);
      }
    }
    d.ctr[(size_t)c * C_COUNT + C_CELL] = 0u;
  }
}

// k == 0 only: preconditioned gradient once lambda_0 is known, |g|^2, and the
// first step length.
__global__ void __launch_bounds__(kThreads) k_precond0(Dev d, int copy0) {
  __shared__ double smd[32];
  __shared__ float2 smc[32];
  __shared__ int flag;
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  CopyState *cs = d.cs + c;
  if (cs->stopped || cs->k != 0) return;
  const float lam = (float)cs->lam;
  const int par = cs->parity;
  const size_t cm = (size_t)c * d.n_mov;
  float g2 = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    const float2 q = d.pa[i];
    float P = fmaxf(1.f, q.x + lam * q.y);
    float gx = (d.gwx[cm + i] + lam * d.gdx[cm + i]) / P;
    float gy = (d.gwy[cm + i] + lam * d.gdy[cm + i]) / P;
    d.g[par][cm + i] = make_float2(gx, gy);
    g2 += gx * gx + gy * gy;
  }
  const double r = block_sum_fc<kThreads>(g2, smc);
  if (threadIdx.x == 0) part_ptr(d, c, S_G2)[blockIdx.x] = r;
  if (!arrive_last(d.ctr + (size_t)c * C_COUNT + C_PRE0, &flag)) return;
  const double s = sum_slot<kThreads>(d, c, S_G2, gridDim.x, smd);
  if (threadIdx.x == 0) {
    advance_scalars(d, cs, true, s, 0.0, 0.0);
    d.ctr[(size_t)c * C_COUNT + C_PRE0] = 0u;
  }
}

// Nesterov step with clamping into the die; the last block closes the
// iteration (k, a_k, buffer parity, max_iters stop).  KEEP_U (backtracking
// on) also saves u_k, and a step that the cell-gradient pass rejected is
// left to k_redo_step.
template <bool KEEP_U>
__global__ void __launch_bounds__(kThreads) k_update(Dev d, int copy0) {
  __shared__ int flag;
  __shared__ float2 smc[32];
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  CopyState *cs = d.cs + c;
  if (cs->stopped) return;
  if constexpr (KEEP_U) {
    if (cs->reject) return;
  }
  const float alpha = (float)cs->alpha, coef = (float)cs->coef;
  const int par = cs->parity;
  const size_t cn = (size_t)c * d.n_cells, cm = (size_t)c * d.n_mov;
  float dv2 = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    const float2 s = d.wh[i];
    const float xh = d.fxh - s.x, yh = d.fyh - s.y;
    const float2 v = d.xy[cn + i];
    const float vx = v.x, vy = v.y;
    const float2 u = d.u[cm + i], g = d.g[par][cm + i];
    const float ux = u.x, uy = u.y;
    float nux = fmaxf(d.fxl, fminf(vx - alpha * g.x, xh));
    float nuy = fmaxf(d.fyl, fminf(vy - alpha * g.y, yh));
    float nvx = fmaxf(d.fxl, fminf(nux + coef * (nux - ux), xh));
    float nvy = fmaxf(d.fyl, fminf(nuy + coef * (nuy - uy), yh));
    if constexpr (KEEP_U) {  // a rejected next step restarts from v_k and u_k
      d.vp[cm + i] = v;
      d.up[cm + i] = u;
    }
    d.u[cm + i] = make_float2(nux, nuy);
    d.xy[cn + i] = make_float2(nvx, nvy);
    const float bx = nvx - vx, by = nvy - vy;
    dv2 += bx * bx + by * by;
  }
  // |v_{k+1} - v_k|^2 per block, for the next iteration's step length: the
  // update knows both points, so v_k need not be stored and read back
  const double r = block_sum_fc<kThreads>(dv2, smc);
  if (threadIdx.x == 0) part_ptr(d, c, S_DV2)[blockIdx.x] = r;
  if (!arrive_last(d.ctr + (size_t)c * C_COUNT + C_UPDATE, &flag)) return;
  if (threadIdx.x == 0) {
    // the iteration's record: its HPWL (WA pass) and overflow at v_k, the
    // step length taken, and the lambda and gamma the next iteration uses
    place_iter_record r;
    r.iter = cs->k;
    r.backtracks = cs->n_back_total;
    r.hpwl_wa = cs->hpwl;
    r.overflow = cs->tau;
    r.lambda = cs->lam;
    r.gamma = cs->gamma;
    r.alpha = cs->alpha;
    d.hist[(size_t)c * d.hist_cap + (cs->n_hist % d.hist_cap)] = r;
    cs->n_hist += 1;
    cs->k += 1;
    cs->a = cs->a_next;
    cs->parity ^= 1;
    if (cs->k >= d.prm.max_iters) cs->stopped = 1;
    d.ctr[(size_t)c * C_COUNT + C_UPDATE] = 0u;
  }
}

// Backtracking: redo the rejected step from v_{k-1}, u_{k-1} and g_{k-1}
// with the shorter length the cell-gradient pass stored; k, a_k and the
// buffer parity stay.  Launched after k_update on handles with backtracking.
__global__ void __launch_bounds__(kThreads) k_redo_step(Dev d, int copy0) {
  __shared__ int flag;
  __shared__ float2 smc[32];
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  CopyState *cs = d.cs + c;
  if (cs->stopped || !cs->reject) return;
  const float alpha = (float)cs->alpha, coef = (float)cs->coef;
  const int par = cs->parity;
  const size_t cn = (size_t)c * d.n_cells, cm = (size_t)c * d.n_mov;
  const float2 *go = d.g[par ^ 1] + cm;
  float dv2 = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    const float2 s = d.wh[i];
    const float xh = d.fxh - s.x, yh = d.fyh - s.y;
    const float2 v = d.vp[cm + i], u = d.up[cm + i], g = go[i];
    const float vx = v.x, vy = v.y, ux = u.x, uy = u.y;
    const float nux = fmaxf(d.fxl, fminf(vx - alpha * g.x, xh));
    const float nuy = fmaxf(d.fyl, fminf(vy - alpha * g.y, yh));
    d.u[cm + i] = make_float2(nux, nuy);
    const float nvx = fmaxf(d.fxl, fminf(nux + coef * (nux - ux), xh));
    const float nvy = fmaxf(d.fyl, fminf(nuy + coef * (nuy - uy), yh));
    d.xy[cn + i] = make_float2(nvx, nvy);
    const float bx = nvx - vx, by = nvy - vy;
    dv2 += bx * bx + by * by;
  }
  const double r = block_sum_fc<kThreads>(dv2, smc);  // the redone step's |v_k - v_{k-1}|^2
  if (threadIdx.x == 0) part_ptr(d, c, S_DV2)[blockIdx.x] = r;
  if (!arrive_last(d.ctr + (size_t)c * C_COUNT + C_UPDATE, &flag)) return;
  if (threadIdx.x == 0) {
    cs->reject = 0;
    d.ctr[(size_t)c * C_COUNT + C_UPDATE] = 0u;
  }
}

// Optimiser reset: clamp the movable positions into the die, u = v, and
// initial scalars (tau_{-1} and gamma_0 follow from the density pass).
__global__ void __launch_bounds__(kThreads) k_reset(Dev d, int copy0) {
  const int c = copy0 + blockIdx.y;
  const size_t cn = (size_t)c * d.n_cells, cm = (size_t)c * d.n_mov;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n_mov; i += gridDim.x * blockDim.x) {
    const float2 v = d.xy[cn + i];
    float vx = fmaxf(d.fxl, fminf(v.x, d.fxh - d.w[i]));
    float vy = fmaxf(d.fyl, fminf(v.y, d.fyh - d.h[i]));
    d.xy[cn + i] = make_float2(vx, vy);
    d.u[cm + i] = make_float2(vx, vy);
    d.gacc[cm + i] = 0ull;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CopyState s = {};
    s.a = 1.0;
    d.cs[c] = s;
  }
}

// Reduce one slot for evaluation calls: d.scal[c * S_COUNT + slot].
__global__ void __launch_bounds__(kRedThreads) k_reduce_slot(Dev d, int slot, int nvals,
                                                             int copy0) {
  __shared__ double sm[32];
  const int c = copy0 + blockIdx.x;
  double s = sum_slot<kRedThreads>(d, c, slot, nvals, sm);
  if (threadIdx.x == 0) d.scal[(size_t)c * S_COUNT + slot] = s;
}

__global__ void k_pack_xy(float2 *dst, const float *x, const float *y, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = make_float2(x[i], y[i]);
}

__global__ void k_unpack_xy(float *x, float *y, const float2 *src, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 v = src[i];
    x[i] = v.x;
    y[i] = v.y;
  }
}

void launch_pack_xy(float2 *dst, const float *x, const float *y, int n, cudaStream_t st) {
  if (n <= 0) return;
  int b = (n + kThreads - 1) / kThreads;
  k_pack_xy<<<b < 4096 ? b : 4096, kThreads, 0, st>>>(dst, x, y, n);
}

void launch_unpack_xy(float *x, float *y, const float2 *src, int n, cudaStream_t st) {
  if (n <= 0) return;
  int b = (n + kThreads - 1) / kThreads;
  k_unpack_xy<<<b < 4096 ? b : 4096, kThreads, 0, st>>>(x, y, src, n);
}

void launch_cell_grad(const Dev &d, int copy0, int ncopy, int eval, cudaStream_t st) {
  if (d.Ms)
    launch_pdl(k_cell_grad<true>, dim3(d.cg_blocks, ncopy), dim3(kThreads), 0, st, d, copy0, eval);
  else
    launch_pdl(k_cell_grad<false>, dim3(d.cg_blocks, ncopy), dim3(kThreads), 0, st, d, copy0, eval);
}
// One failing index check and no access (place_test_bounds_check).
__global__ void k_test_bounds(Dev d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const long long i = d.n_cells;  // one past the last cell
    if (HP_IN(d.err, i, d.n_cells, BS_WA_CELL)) d.err[1] = 0;  // (reached only when it passes)
  }
}
void launch_test_bounds(const Dev &d, cudaStream_t st) { k_test_bounds<<<1, 32, 0, st>>>(d); }

int cell_grad_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cell_grad<false>, kThreads, 0) != cudaSuccess || n < 1)
    n = 1;
  return n;
}
void launch_precond0(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  launch_pdl(k_precond0, dim3(d.cell_blocks, ncopy), dim3(kThreads), 0, st, d, copy0);
}
void launch_update(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  const dim3 grid(d.cell_blocks, ncopy);
  if (d.up) {
    launch_pdl(k_update<true>, grid, dim3(kThreads), 0, st, d, copy0);
    launch_pdl(k_redo_step, grid, dim3(kThreads), 0, st, d, copy0);
  } else {
    launch_pdl(k_update<false>, grid, dim3(kThreads), 0, st, d, copy0);
  }
}
void launch_reset(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  k_reset<<<dim3(d.cell_blocks, ncopy), kThreads, 0, st>>>(d, copy0);
}
void launch_reduce_slot(const Dev &d, int slot, int nvals, int copy0, int ncopy,
                        cudaStream_t st) {
  k_reduce_slot<<<ncopy, kRedThreads, 0, st>>>(d, slot, nvals, copy0);
}

}  // namespace hp
