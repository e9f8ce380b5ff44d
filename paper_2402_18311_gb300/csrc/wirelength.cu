// Weighted-average wirelength (Eq. 3) and its gradient, and the exact FP64
// HPWL (Eq. 1).
//
// For one net and one axis with pin coordinates p_j, m+ = max p, m- = min p,
// a_j = exp((p_j - m+)/g), b_j = exp((m- - p_j)/g), S+ = sum a,
// R+ = sum (p_j - m+) a_j / S+, S- = sum b, R- = sum (p_j - m-) b_j / S-:
//   WL_e = (m+ - m-) + R+ - R-                     (Eq. 3, exactly)
//   dWL_e/dp_j = (a_j/S+)(1 + (p_j - m+ - R+)/g) - (b_j/S-)(1 - (p_j - m- - R-)/g)
// Pin coordinates are taken relative to the net's first pin (WA is
// shift-invariant), (x_j - x_0) + (dx_j - dx_0), and exponents relative to
// m+ / m-, so FP32 keeps the digits that matter even where the cells of a
// net sit close together far from the origin.
//
// Exponentials use the fast intrinsic __expf.  Its documented error grows
// with |argument| (2 + floor(|1.16 x|) ulp); every argument here is <= 0 after
// the max/min shift, and the terms with large |x| are the ones that vanish in
// the sums, so the WA value and gradient stay well inside their tolerance.
//
// Nets are grouped by degree at create: one thread per net up to 4 pins,
// groups of 4 lanes up to 16 pins, 16 lanes up to 64, a warp up to 256 (the
// pins of these nets stay in registers, 4 or 8 per lane), and a block of 256
// threads beyond, which keeps the coordinates of up to 3072 of the net's pins
// in shared memory between its three passes.  Positions are interleaved
// (x, y), so every pin costs one gather.  Each pin's gradient is
// added to its cell as a packed fixed-point integer (add_pin_grad): one
// 64-bit reduction per pin into an array that stays in L2, no floating-point
// atomics, deterministic results.
#include <cfloat>
#include <mutex>

#include "common.cuh"
#include "internal.cuh"

namespace hp {

template <int G>
__device__ __forceinline__ float gmax(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <int G>
__device__ __forceinline__ float gmin(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <int G>
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float copy_gamma(const Dev &d, int c, const float *ovr) {
  return ovr ? *ovr : (float)d.cs[c].gamma;
}

// The arithmetic of Eq. 3 per pin and per net, every operation written with
// its rounding (no multiply-add left for the compiler to contract or not), so
// that every build of the library computes the same bits.
//   sums:     S+ += a, T+ += (p - m+) a, S- += b, T- += (p - m-) b
//   gradient: (a/S+)(1 + (p - m+ - R+)/g) - (b/S-)(1 - (p - m- - R-)/g)
__device__ __forceinline__ void wa_sums(float p, float mx, float mn, float ig, float &sp, float &tp,
                                        float &sm, float &tm) {
  const float dp = __fsub_rn(p, mx), dm = __fsub_rn(p, mn);
  const float a = __expf(__fmul_rn(dp, ig)), b = __expf(__fmul_rn(__fsub_rn(mn, p), ig));
  sp = __fadd_rn(sp, a);
  tp = __fmaf_rn(dp, a, tp);
  sm = __fadd_rn(sm, b);
  tm = __fmaf_rn(dm, b, tm);
}
__device__ __forceinline__ float wa_grad(float p, float mx, float mn, float ig, float isp, float ism,
                                         float rp, float rm) {
  const float dp = __fsub_rn(p, mx), dm = __fsub_rn(p, mn);
  const float a = __expf(__fmul_rn(dp, ig)), b = __expf(__fmul_rn(__fsub_rn(mn, p), ig));
  const float fp = __fmaf_rn(__fsub_rn(dp, rp), ig, 1.f);
  const float fm = __fmaf_rn(-__fsub_rn(dm, rm), ig, 1.f);
  return __fmaf_rn(__fmul_rn(a, isp), fp, -__fmul_rn(__fmul_rn(b, ism), fm));
}
// a net's HPWL (its pin extents) and WA value, weighted, into the thread's sums
__device__ __forceinline__ void wa_net_sums(float wn, float mxx, float mnx, float mxy, float mny,
                                            float rxp, float rxm, float ryp, float rym,
                                            float &hp_acc, float &wl_acc) {
  const float ex = __fsub_rn(mxx, mnx), ey = __fsub_rn(mxy, mny);
  hp_acc = __fmaf_rn(wn, __fadd_rn(ex, ey), hp_acc);
  wl_acc = __fmaf_rn(wn, __fadd_rn(__fadd_rn(ex, __fsub_rn(rxp, rxm)), __fadd_rn(ey, __fsub_rn(ryp, rym))),
                     wl_acc);
}

// One net of deg <= D pins on one thread, pins held in registers, no shuffles.
template <int D>
__device__ __forceinline__ void wa_net_small(const Dev &d, const float2 *xy, unsigned long long *ga,
                                             int e, int p0, int deg, float ig, float &hp_acc,
                                             float &wl_acc) {
    int cell[D];
    float2 off[D], pos[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k < deg) {
        cell[k] = d.pin_cell[p0 + k];
        HP_FIX(d.err, cell[k], d.n_cells, BS_WA_CELL);
        off[k] = d.pin_off[p0 + k];
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < deg) pos[k] = xy[cell[k]];
    float px[D], py[D];
    px[0] = 0.f;
    py[0] = 0.f;
#pragma unroll
    for (int k = 1; k < D; ++k) {
      if (k < deg) {
        px[k] = (pos[k].x - pos[0].x) + (off[k].x - off[0].x);
        py[k] = (pos[k].y - pos[0].y) + (off[k].y - off[0].y);
      }
    }
    float mxx = 0.f, mnx = 0.f, mxy = 0.f, mny = 0.f;
#pragma unroll
    for (int k = 1; k < D; ++k) {
      if (k < deg) {
        mxx = fmaxf(mxx, px[k]); mnx = fminf(mnx, px[k]);
        mxy = fmaxf(mxy, py[k]); mny = fminf(mny, py[k]);
      }
    }
    float sxp = 0.f, txp = 0.f, sxm = 0.f, txm = 0.f, syp = 0.f, typ = 0.f, sym = 0.f, tym = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k < deg) {
        wa_sums(px[k], mxx, mnx, ig, sxp, txp, sxm, txm);
        wa_sums(py[k], mxy, mny, ig, syp, typ, sym, tym);
      }
    }
    const float wn = d.net_w ? d.net_w[e] : 1.0f;
    const float isxp = 1.f / sxp, isxm = 1.f / sxm, isyp = 1.f / syp, isym = 1.f / sym;
    const float rxp = txp * isxp, rxm = txm * isxm, ryp = typ * isyp, rym = tym * isym;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k < deg) {
        const float gx = wa_grad(px[k], mxx, mnx, ig, isxp, isxm, rxp, rxm);
        const float gy = wa_grad(py[k], mxy, mny, ig, isyp, isym, ryp, rym);
        add_pin_grad(d, ga, cell[k], __fmul_rn(gx, wn), __fmul_rn(gy, wn));
      }
    }
    wa_net_sums(wn, mxx, mnx, mxy, mny, rxp, rxm, ryp, rym, hp_acc, wl_acc);
}

// One 2-pin net in closed form.  Per axis, with d the second pin's
// coordinate relative to the first, Eq. 3 reduces to
//   WL = |d| tanh(|d| / 2g),  dWL/dp_1 = -dWL/dp_0 = sign(d) (th + (|d|/2g)(1 - th^2)),
// th = tanh(|d|/2g) = (1 - t)/(1 + t) with t = exp(-|d|/g): one exponential
// per axis instead of eight.  For |d| << g the difference 1 - t loses
// relative digits, but the value and the gradient it feeds are then of
// order |d|/g, far below the other terms of the sums they enter.
// Every operation is written with its rounding (no contraction left to the
// compiler), so the result is the same in every build of the library.
__device__ __forceinline__ void wa_axis_2pin(float dd, float ig, float &wl, float &gr) {
  const float ad = fabsf(dd);
  const float u = __fmul_rn(ad, ig);
  const float t = __expf(-u);
  const float th = __fdiv_rn(__fsub_rn(1.f, t), __fadd_rn(1.f, t));
  wl = __fmul_rn(ad, th);
  gr = copysignf(__fmaf_rn(__fmul_rn(0.5f, u), __fmaf_rn(-th, th, 1.f), th), dd);
}

__device__ __forceinline__ void wa_net_2pin(const Dev &d, const float2 *xy, unsigned long long *ga,
                                            int e, int p0, float ig, float &hp_acc, float &wl_acc) {
  int c0 = d.pin_cell[p0], c1 = d.pin_cell[p0 + 1];
  HP_FIX(d.err, c0, d.n_cells, BS_WA_CELL);
  HP_FIX(d.err, c1, d.n_cells, BS_WA_CELL);
  const float2 o0 = d.pin_off[p0], o1 = d.pin_off[p0 + 1];
  const float2 v0 = xy[c0], v1 = xy[c1];
  const float dx = (v1.x - v0.x) + (o1.x - o0.x), dy = (v1.y - v0.y) + (o1.y - o0.y);
  float wx, gx, wy, gy;
  wa_axis_2pin(dx, ig, wx, gx);
  wa_axis_2pin(dy, ig, wy, gy);
  const float wn = d.net_w ? d.net_w[e] : 1.0f;
  const float gxw = __fmul_rn(gx, wn), gyw = __fmul_rn(gy, wn);
  add_pin_grad(d, ga, c0, -gxw, -gyw);
  add_pin_grad(d, ga, c1, gxw, gyw);
  hp_acc = __fmaf_rn(wn, __fadd_rn(fabsf(dx), fabsf(dy)), hp_acc);
  wl_acc = __fmaf_rn(wn, __fadd_rn(wx, wy), wl_acc);
}

// Nets of at most D pins: one thread per net.  The class is ordered by
// degree, so a warp's nets share one path: the closed form for 2 pins (most
// nets of a netlist), the unrolled general form otherwise (a third path for
// 3-pin nets made the kernel spill and was slower).
template <int D>
__global__ void __launch_bounds__(kThreads, 4) k_wa_thread(Dev d, int copy0, int cls, int eval,
                                                            const float *gamma_ovr) {
  __shared__ float2 sm[32];
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  const float g = copy_gamma(d, c, gamma_ovr);
  const float ig = 1.0f / g;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  unsigned long long *ga = d.gacc + (size_t)c * d.n_mov;
  const int e_end = d.cls_begin[cls + 1];
  // each thread sums its few nets in FP32; the block sum is compensated (the
  // HPWL sum drives the lambda schedule through differences of consecutive
  // iterations)
  float hp_acc = 0.f, wl_acc = 0.f;
  for (int e = d.cls_begin[cls] + blockIdx.x * blockDim.x + threadIdx.x; e < e_end;
       e += gridDim.x * blockDim.x) {
    const int p0 = d.net_ptr[e], p1 = d.net_ptr[e + 1];
    const int deg = p1 - p0;
    if (deg <= 0) continue;
    if (!HP_IN(d.err, p0, d.n_pins, BS_WA_PIN) || !HP_IN(d.err, p1, d.n_pins + 1, BS_WA_PIN) ||
        !HP_IN(d.err, deg, D + 1, BS_WA_PIN))
      continue;
    if (deg == 2)
      wa_net_2pin(d, xy, ga, e, p0, ig, hp_acc, wl_acc);
    else
      wa_net_small<D>(d, xy, ga, e, p0, deg, ig, hp_acc, wl_acc);
  }
  const double rh = block_sum_fc<kThreads>(hp_acc, sm);
  const double rw = block_sum_fc<kThreads>(wl_acc, sm);
  if (threadIdx.x == 0) {
    size_t base = (size_t)c * S_COUNT * d.nb_red + d.wa_block_base[cls] + blockIdx.x;
    d.part[base + (size_t)S_HPWL * d.nb_red] = rh;
    d.part[base + (size_t)S_WL * d.nb_red] = rw;
  }
}

// One net of at most G * PPL pins on G lanes (lane = this thread's lane in
// its group), each lane holding up to PPL of the net's pins in registers, so
// every pin is gathered once.  valid: the group has a net (all G lanes of a
// group agree).
template <int G, int PPL>
__device__ __forceinline__ void wa_group_net(const Dev &d, const float2 *xy, unsigned long long *ga,
                                             int e, bool valid, int lane, float ig, float &hp_acc,
                                             float &wl_acc) {
    int p0 = 0, p1 = 0;
    if (valid) {
      p0 = d.net_ptr[e];
      p1 = d.net_ptr[e + 1];
      if (!HP_IN(d.err, p0, d.n_pins + 1, BS_WA_PIN) || !HP_IN(d.err, p1, d.n_pins + 1, BS_WA_PIN) ||
          !HP_IN(d.err, p1 - p0, G * PPL + 1, BS_WA_PIN))
        p0 = p1 = 0;
    }
    const float wn = (valid && d.net_w) ? d.net_w[e] : 1.0f;
    // all of the net's loads in flight together; coordinates relative to the
    // net's first pin, (x_j - x_0) + (dx_j - dx_0), round relative to the pin
    // spacing, not to the absolute position
    int cl[PPL];
    float2 of[PPL], v[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int j = p0 + lane + k * G;
      cl[k] = j < p1 ? d.pin_cell[j] : -1;
      if (cl[k] >= 0) HP_FIX(d.err, cl[k], d.n_cells, BS_WA_CELL);
      of[k] = j < p1 ? d.pin_off[j] : make_float2(0.f, 0.f);
    }
    float2 r0 = make_float2(0.f, 0.f), o0 = make_float2(0.f, 0.f);
    if (p1 > p0) {
      o0 = d.pin_off[p0];
      int c0 = d.pin_cell[p0];
      HP_FIX(d.err, c0, d.n_cells, BS_WA_CELL);
      r0 = xy[c0];
    }
#pragma unroll
    for (int k = 0; k < PPL; ++k) v[k] = cl[k] >= 0 ? xy[cl[k]] : make_float2(0.f, 0.f);
    float px[PPL], py[PPL];
    float mxx = -FLT_MAX, mnx = FLT_MAX, mxy = -FLT_MAX, mny = FLT_MAX;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      px[k] = (v[k].x - r0.x) + (of[k].x - o0.x);
      py[k] = (v[k].y - r0.y) + (of[k].y - o0.y);
      if (cl[k] >= 0) {
        mxx = fmaxf(mxx, px[k]); mnx = fminf(mnx, px[k]);
        mxy = fmaxf(mxy, py[k]); mny = fminf(mny, py[k]);
      }
    }
    mxx = gmax<G>(mxx); mnx = gmin<G>(mnx);
    mxy = gmax<G>(mxy); mny = gmin<G>(mny);
    float sxp = 0.f, txp = 0.f, sxm = 0.f, txm = 0.f;
    float syp = 0.f, typ = 0.f, sym = 0.f, tym = 0.f;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      if (cl[k] >= 0) {
        wa_sums(px[k], mxx, mnx, ig, sxp, txp, sxm, txm);
        wa_sums(py[k], mxy, mny, ig, syp, typ, sym, tym);
      }
    }
    sxp = gsum<G>(sxp); txp = gsum<G>(txp); sxm = gsum<G>(sxm); txm = gsum<G>(txm);
    syp = gsum<G>(syp); typ = gsum<G>(typ); sym = gsum<G>(sym); tym = gsum<G>(tym);
    if (p1 > p0) {
      const float isxp = 1.f / sxp, isxm = 1.f / sxm, isyp = 1.f / syp, isym = 1.f / sym;
      const float rxp = txp * isxp, rxm = txm * isxm, ryp = typ * isyp, rym = tym * isym;
#pragma unroll
      for (int k = 0; k < PPL; ++k) {
        if (cl[k] >= 0) {
          const float gx = wa_grad(px[k], mxx, mnx, ig, isxp, isxm, rxp, rxm);
          const float gy = wa_grad(py[k], mxy, mny, ig, isyp, isym, ryp, rym);
          add_pin_grad(d, ga, cl[k], __fmul_rn(gx, wn), __fmul_rn(gy, wn));
        }
      }
      if (lane == 0) wa_net_sums(wn, mxx, mnx, mxy, mny, rxp, rxm, ryp, rym, hp_acc, wl_acc);
    }
  }

// Nets of a degree class in two sub-ranges, the class ordered so that the
// nets of at most GL * PPL pins come first (up to d.cls_split[cls]): those
// on GL lanes each, the rest on G lanes.  A warp takes 32 / GL or 32 / G
// consecutive nets of one sub-range, so the choice is warp-uniform and no
// lane slot is spent on the short nets' empty halves.  MINB resident blocks
// per SM bound the registers (no spills at the chosen values).
template <int G, int GL, int PPL, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_wa_group(Dev d, int copy0, int cls, int eval,
                                                        const float *gamma_ovr) {
  __shared__ float2 sm[32];
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  const float g = copy_gamma(d, c, gamma_ovr);
  const float ig = 1.0f / g;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  unsigned long long *ga = d.gacc + (size_t)c * d.n_mov;
  const int e_beg = d.cls_begin[cls], e_mid = d.cls_split[cls], e_end = d.cls_begin[cls + 1];
  constexpr int NL = 32 / GL, NH = 32 / G;  // nets per warp task in each sub-range
  const int tlo = (e_mid - e_beg + NL - 1) / NL;
  const int tall = tlo + (e_end - e_mid + NH - 1) / NH;
  const int wl = threadIdx.x & 31;
  const int nwarps = gridDim.x * (kThreads / 32);
  float hp_acc = 0.f, wl_acc = 0.f;
  for (int t = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); t < tall; t += nwarps) {
    if (t < tlo) {
      const int e = e_beg + t * NL + wl / GL;
      wa_group_net<GL, PPL>(d, xy, ga, e, e < e_mid, wl % GL, ig, hp_acc, wl_acc);
    } else {
      const int e = e_mid + (t - tlo) * NH + wl / G;
      wa_group_net<G, PPL>(d, xy, ga, e, e < e_end, wl % G, ig, hp_acc, wl_acc);
    }
  }
  const double rh = block_sum_fc<kThreads>(hp_acc, sm);
  const double rw = block_sum_fc<kThreads>(wl_acc, sm);
  if (threadIdx.x == 0) {
    size_t base = (size_t)c * S_COUNT * d.nb_red + d.wa_block_base[cls] + blockIdx.x;
    d.part[base + (size_t)S_HPWL * d.nb_red] = rh;
    d.part[base + (size_t)S_WL * d.nb_red] = rw;
  }
}

// Block-wide reductions for the one-block-per-net kernel: N values per
// thread, maxima or sums, in a fixed order, the results in every thread.
constexpr int kBigNet = 256;
constexpr int kBigWarps = kBigNet / 32;
template <int N, bool MAX>
__device__ __forceinline__ void block_all(float (&v)[N], float *sm) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float w = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = MAX ? fmaxf(v[k], w) : v[k] + w;
    }
  }
  __syncthreads();  // the previous readers of sm are done
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) sm[(threadIdx.x >> 5) * N + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float r = sm[k];
#pragma unroll
    for (int i = 1; i < kBigWarps; ++i) r = MAX ? fmaxf(r, sm[i * N + k]) : r + sm[i * N + k];
    v[k] = r;
  }
}

// One block per net (degree > 256), the nets in descending degree so the
// longest start first.  The net-relative coordinates of a net's first `cap`
// pins stay in dynamic shared memory between the three passes; pins beyond
// `cap` are gathered again in each pass.  A small cap keeps more blocks
// resident, which matters more than the re-gathers of the longest nets.
__global__ void __launch_bounds__(kBigNet) k_wa_big(Dev d, int copy0, int cls, int eval,
                                                    const float *gamma_ovr, int cap) {
  extern __shared__ float dyn[];
  float *spx = dyn, *spy = dyn + cap;
  __shared__ float sm[kBigWarps * 8];
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  const float g = copy_gamma(d, c, gamma_ovr);
  const float ig = 1.0f / g;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  unsigned long long *ga = d.gacc + (size_t)c * d.n_mov;
  double hp_acc = 0.0, wl_acc = 0.0;
  for (int e = d.cls_begin[cls] + blockIdx.x; e < d.cls_begin[cls + 1]; e += gridDim.x) {
    const int p0 = d.net_ptr[e], p1 = d.net_ptr[e + 1];
    // (every thread of the block tests the same net, so a skip is uniform)
    if (!HP_IN(d.err, p0, d.n_pins, BS_WA_PIN) || !HP_IN(d.err, p1, d.n_pins + 1, BS_WA_PIN) ||
        !HP_IN(d.err, p1 - p0, 1 << 30, BS_WA_PIN))
      continue;
    const float wn = d.net_w ? d.net_w[e] : 1.0f;
    const float2 o0 = d.pin_off[p0];
    int c0 = d.pin_cell[p0];
    HP_FIX(d.err, c0, d.n_cells, BS_WA_CELL);
    const float2 v0 = xy[c0];
    const float rx = v0.x, ry = v0.y, rdx = o0.x, rdy = o0.y;
    float ext[4] = {-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};  // max x, -min x, max y, -min y
#pragma unroll 4
    for (int j = p0 + threadIdx.x; j < p1; j += kBigNet) {
      const float2 o = d.pin_off[j];
      int cj = d.pin_cell[j];
      HP_FIX(d.err, cj, d.n_cells, BS_WA_CELL);
      const float2 v = xy[cj];
      const float px = (v.x - rx) + (o.x - rdx), py = (v.y - ry) + (o.y - rdy);
      if (j - p0 < cap) { spx[j - p0] = px; spy[j - p0] = py; }
      ext[0] = fmaxf(ext[0], px); ext[1] = fmaxf(ext[1], -px);
      ext[2] = fmaxf(ext[2], py); ext[3] = fmaxf(ext[3], -py);
    }
    block_all<4, true>(ext, sm);
    const float mxx = ext[0], mnx = -ext[1], mxy = ext[2], mny = -ext[3];
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int j = p0 + threadIdx.x; j < p1; j += kBigNet) {
      float px, py;
      if (j - p0 < cap) {
        px = spx[j - p0]; py = spy[j - p0];
      } else {
        const float2 o = d.pin_off[j];
        int cj = d.pin_cell[j];
        HP_FIX(d.err, cj, d.n_cells, BS_WA_CELL);
        const float2 v = xy[cj];
        px = (v.x - rx) + (o.x - rdx); py = (v.y - ry) + (o.y - rdy);
      }
      wa_sums(px, mxx, mnx, ig, s[0], s[1], s[2], s[3]);
      wa_sums(py, mxy, mny, ig, s[4], s[5], s[6], s[7]);
    }
    block_all<8, false>(s, sm);
    const float isxp = 1.f / s[0], isxm = 1.f / s[2], isyp = 1.f / s[4], isym = 1.f / s[6];
    const float rxp = s[1] * isxp, rxm = s[3] * isxm, ryp = s[5] * isyp, rym = s[7] * isym;
#pragma unroll 4
    for (int j = p0 + threadIdx.x; j < p1; j += kBigNet) {
      float px, py;
      int cj = d.pin_cell[j];
      HP_FIX(d.err, cj, d.n_cells, BS_WA_CELL);
      if (j - p0 < cap) {
        px = spx[j - p0]; py = spy[j - p0];
      } else {
        const float2 o = d.pin_off[j];
        const float2 v = xy[cj];
        px = (v.x - rx) + (o.x - rdx); py = (v.y - ry) + (o.y - rdy);
      }
      const float gx = wa_grad(px, mxx, mnx, ig, isxp, isxm, rxp, rxm);
      const float gy = wa_grad(py, mxy, mny, ig, isyp, isym, ryp, rym);
      add_pin_grad(d, ga, cj, __fmul_rn(gx, wn), __fmul_rn(gy, wn));
    }
    hp_acc += wn * ((mxx - mnx) + (mxy - mny));
    wl_acc += wn * (((mxx - mnx) + (rxp - rxm)) + ((mxy - mny) + (ryp - rym)));
    __syncthreads();  // the shared pin cache is reused by the next net
  }
  if (threadIdx.x == 0) {
    size_t base = (size_t)c * S_COUNT * d.nb_red + d.wa_block_base[cls] + blockIdx.x;
    d.part[base + (size_t)S_HPWL * d.nb_red] = hp_acc;
    d.part[base + (size_t)S_WL * d.nb_red] = wl_acc;
  }
}

// Exact HPWL (Eq. 1) in FP64: pin coordinates are widened from the FP32
// position and offset before they are added, so every pin coordinate, max and
// min is exact; only the sum over nets rounds.  G lanes per net (whole
// warps loop over long nets).
template <int G>
__global__ void __launch_bounds__(kThreads) k_hpwl64(Dev d, int copy0, int e_begin, int e_end,
                                                      int slot_base) {
  __shared__ double sm[32];
  const int c = copy0 + blockIdx.y;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  constexpr int NPB = kThreads / G;
  const int lane = threadIdx.x % G;
  double acc = 0.0;
  for (int base = e_begin + blockIdx.x * NPB; base < e_end; base += gridDim.x * NPB) {
    const int e = base + threadIdx.x / G;
    int p0 = 0, p1 = 0;
    if (e < e_end) {
      p0 = d.net_ptr[e];
      p1 = d.net_ptr[e + 1];
      if (!HP_IN(d.err, p0, d.n_pins + 1, BS_HPWL_PIN) || !HP_IN(d.err, p1, d.n_pins + 1, BS_HPWL_PIN))
        p0 = p1 = 0;
    }
    double mxx = -1e300, mnx = 1e300, mxy = -1e300, mny = 1e300;
    for (int j = p0 + lane; j < p1; j += G) {
      const float2 o = d.pin_off[j];
      int cj = d.pin_cell[j];
      HP_FIX(d.err, cj, d.n_cells, BS_HPWL_CELL);
      const float2 v = xy[cj];
      double px = (double)v.x + (double)o.x, py = (double)v.y + (double)o.y;
      mxx = fmax(mxx, px); mnx = fmin(mnx, px);
      mxy = fmax(mxy, py); mny = fmin(mny, py);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      mxx = fmax(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
      mnx = fmin(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
      mxy = fmax(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
      mny = fmin(mny, __shfl_xor_sync(0xffffffffu, mny, o));
    }
    if (lane == 0 && p1 > p0) {
      double wn = d.net_w ? (double)d.net_w[e] : 1.0;
      acc += wn * ((mxx - mnx) + (mxy - mny));
    }
  }
  double r = block_sum<kThreads>(acc, sm);
  if (threadIdx.x == 0)
    d.part[((size_t)c * S_COUNT + S_HP64) * d.nb_red + slot_base + blockIdx.x] = r;
}

// One degree class's kernel; pdl: launched programmatically after the
// kernel before it in the stream.
static void launch_wa_one(const Dev &d, int cls, int copy0, int ncopy, int eval,
                          const float *gamma_ovr, bool pdl, cudaStream_t st) {
  const dim3 grid(d.wa_blocks[cls], ncopy), blk(kThreads);
  switch (cls) {
    case 0:
      if (pdl) launch_pdl(k_wa_thread<4>, grid, blk, 0, st, d, copy0, cls, eval, gamma_ovr);
      else k_wa_thread<4><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr);
      break;
    case 1:
      if (pdl) launch_pdl(k_wa_group<4, 2, 4, 5>, grid, blk, 0, st, d, copy0, cls, eval, gamma_ovr);
      else k_wa_group<4, 2, 4, 5><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr);
      break;
    case 2:
      if (pdl) launch_pdl(k_wa_group<16, 8, 4, 5>, grid, blk, 0, st, d, copy0, cls, eval, gamma_ovr);
      else k_wa_group<16, 8, 4, 5><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr);
      break;
    case 3:
      if (pdl) launch_pdl(k_wa_group<32, 32, 8, 1>, grid, blk, 0, st, d, copy0, cls, eval, gamma_ovr);
      else k_wa_group<32, 32, 8, 1><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr);
      break;
    default: {
      const size_t sm = 2 * sizeof(float) * d.wa_big_cap;
      if (pdl)
        launch_pdl(k_wa_big, grid, dim3(kBigNet), sm, st, d, copy0, cls, eval, gamma_ovr,
                   d.wa_big_cap);
      else
        k_wa_big<<<grid, kBigNet, sm, st>>>(d, copy0, cls, eval, gamma_ovr, d.wa_big_cap);
      break;
    }
  }
}

void launch_wa(const Dev &d, int copy0, int ncopy, int eval, const float *gamma_ovr,
               cudaStream_t st) {
  int launched = 0;
  for (int cls = 0; cls < d.n_cls; ++cls) {
    if (d.wa_blocks[cls] == 0) continue;
    // the first class follows whatever precedes it in the stream (an event
    // or a copy); the others follow a WA kernel and launch programmatically
    launch_wa_one(d, cls, copy0, ncopy, eval, gamma_ovr, launched++ > 0, st);
  }
}

// Branch of each degree class (thread, 4-lane, 16-lane, warp, big) for 1, 2
// and 3 branches.  Two: the short nets beside the long ones; three: the
// thread class alone, the group classes, the warp and big-net classes (whose
// few long blocks then overlap the others' many short ones).
constexpr int kWaBranch[3][5] = {{0, 0, 0, 0, 0}, {0, 0, 1, 1, 1}, {0, 1, 1, 2, 2}};

void launch_wa_branches(const Dev &d, int copy0, int ncopy, const cudaStream_t *st) {
  const int nb = d.wa_streams < 1 ? 1 : (d.wa_streams > kMaxWaStreams ? kMaxWaStreams : d.wa_streams);
  int launched[kMaxWaStreams] = {0, 0, 0};
  for (int cls = 0; cls < d.n_cls; ++cls) {
    if (d.wa_blocks[cls] == 0) continue;
    const int b = kWaBranch[nb - 1][cls < 5 ? cls : 4];
    // the first class of a branch follows the branch's fork; the others
    // follow a WA kernel and launch programmatically
    launch_wa_one(d, cls, copy0, ncopy, 0, nullptr, launched[b]++ > 0, st[b]);
  }
}

void launch_wa_class(const Dev &d, int cls, int copy0, int ncopy, int eval, cudaStream_t st) {
  if (cls >= 0 && cls < d.n_cls && d.wa_blocks[cls] > 0)
    launch_wa_one(d, cls, copy0, ncopy, eval, nullptr, false, st);
}

// The big-net kernel's dynamic shared-memory limit is a property of the
// function, shared by every handle in the process: it only ever grows.
int wa_prepare(int cap) {
  static std::mutex mu;
  static int granted = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (cap <= granted) return 0;
  cudaError_t e = cudaFuncSetAttribute(k_wa_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * sizeof(float) * cap));
  if (e != cudaSuccess) return -1;
  granted = cap;
  return 0;
}

// Nets above 256 pins: one block per net, FP64 block reductions.
__global__ void __launch_bounds__(kThreads) k_hpwl64_big(Dev d, int copy0, int e_begin, int e_end,
                                                          int slot_base) {
  __shared__ double sm[4][32];
  const int c = copy0 + blockIdx.y;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  double acc = 0.0;
  for (int e = e_begin + blockIdx.x; e < e_end; e += gridDim.x) {
    int p0 = d.net_ptr[e], p1 = d.net_ptr[e + 1];
    if (!HP_IN(d.err, p0, d.n_pins + 1, BS_HPWL_PIN) || !HP_IN(d.err, p1, d.n_pins + 1, BS_HPWL_PIN))
      p0 = p1 = 0;
    double v[4] = {-1e300, -1e300, -1e300, -1e300};  // max x, -min x, max y, -min y
    for (int j = p0 + threadIdx.x; j < p1; j += kThreads) {
      const float2 o = d.pin_off[j];
      int cj = d.pin_cell[j];
      HP_FIX(d.err, cj, d.n_cells, BS_HPWL_CELL);
      const float2 q = xy[cj];
      const double px = (double)q.x + (double)o.x, py = (double)q.y + (double)o.y;
      v[0] = fmax(v[0], px); v[1] = fmax(v[1], -px);
      v[2] = fmax(v[2], py); v[3] = fmax(v[3], -py);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] = fmax(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
      for (int k = 0; k < 4; ++k) sm[k][threadIdx.x >> 5] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
      double r[4];
      for (int k = 0; k < 4; ++k) {
        r[k] = sm[k][0];
        for (int w = 1; w < kThreads / 32; ++w) r[k] = fmax(r[k], sm[k][w]);
      }
      const double wn = d.net_w ? (double)d.net_w[e] : 1.0;
      acc += wn * ((r[0] + r[1]) + (r[2] + r[3]));
    }
  }
  if (threadIdx.x == 0)
    d.part[((size_t)c * S_COUNT + S_HP64) * d.nb_red + slot_base + blockIdx.x] = acc;
}

// Measurement kernel: only the memory operations the WA pass cannot avoid
// on this netlist, with nothing else in the way.  Per pin it reads pin_cell
// and the offsets (streamed), gathers the cell's position (random 8 bytes)
// and adds one packed 64-bit value to the cell's gradient sum (random
// reduction); per net it reads net_ptr.  Pin-parallel, eight pins per
// thread with all gathers in flight before the reductions.  Its time is the
// floor of the WA stage's gather-and-reduce traffic on this index stream.
constexpr int kFloorPins = 8;
__global__ void __launch_bounds__(kThreads) k_wa_floor(Dev d, int copy0) {
  pdl_wait();
  const int c = copy0 + blockIdx.y;
  const float2 *xy = d.xy + (size_t)c * d.n_cells;
  unsigned long long *ga = d.gacc + (size_t)c * d.n_mov;
  const int P = d.n_pins;
  const int stride = gridDim.x * blockDim.x * kFloorPins;
  for (int j0 = (blockIdx.x * blockDim.x) * kFloorPins + threadIdx.x; j0 < P; j0 += stride) {
    int cl[kFloorPins];
    float2 of[kFloorPins], v[kFloorPins];
#pragma unroll
    for (int k = 0; k < kFloorPins; ++k) {
      const int j = j0 + k * blockDim.x;
      cl[k] = j < P ? d.pin_cell[j] : -1;
      of[k] = j < P ? d.pin_off[j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < kFloorPins; ++k) v[k] = cl[k] >= 0 ? xy[cl[k]] : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kFloorPins; ++k)
      if (cl[k] >= 0) add_pin_grad(d, ga, cl[k], (v[k].x + of[k].x) * 1e-6f, (v[k].y + of[k].y) * 1e-6f);
  }
  // net_ptr, streamed once
  int acc = 0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= d.n_nets; e += gridDim.x * blockDim.x)
    acc ^= d.net_ptr[e];
  if (acc == 0x7fffffff) d.err[1] = acc;  // keeps the loads; never true for a valid netlist
}

void launch_wa_floor(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  const int per_block = kThreads * kFloorPins;
  int nb = (d.n_pins + per_block - 1) / per_block;
  nb = nb < 1 ? 1 : (nb > kMaxCellBlocks ? kMaxCellBlocks : nb);
  k_wa_floor<<<dim3(nb, ncopy), kThreads, 0, st>>>(d, copy0);
}

int hpwl64_blocks(const Dev &d) { return 2 * d.cell_blocks; }

void launch_hpwl64(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  // nets up to 4 pins: 4 lanes each; up to 256 pins: a warp each; longer: a block each
  const int split = d.cls_begin[1], big = d.cls_begin[4];
  const int half = d.cell_blocks / 2 > 0 ? d.cell_blocks / 2 : 1;
  dim3 grid(d.cell_blocks, ncopy), grid2(half, ncopy);
  k_hpwl64<4><<<grid, kThreads, 0, st>>>(d, copy0, 0, split, 0);
  k_hpwl64<32><<<grid2, kThreads, 0, st>>>(d, copy0, split, big, d.cell_blocks);
  k_hpwl64_big<<<grid2, kThreads, 0, st>>>(d, copy0, big, d.n_nets, d.cell_blocks + half);
}

}  // namespace hp
