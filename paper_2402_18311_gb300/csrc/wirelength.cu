// Weighted-average wirelength (Eq. 3) and its gradient, and the exact FP64
// HPWL (Eq. 1).
//
// For one net and one axis with pin coordinates p_j, m+ = max p, m- = min p,
// a_j = exp((p_j - m+)/g), b_j = exp((m- - p_j)/g), S+ = sum a,
// R+ = sum (p_j - m+) a_j / S+, S- = sum b, R- = sum (p_j - m-) b_j / S-:
//   WL_e = (m+ - m-) + R+ - R-                     (Eq. 3, exactly)
//   dWL_e/dp_j = (a_j/S+)(1 + (p_j - m+ - R+)/g) - (b_j/S-)(1 - (p_j - m- - R-)/g)
// Pin coordinates are taken relative to the net's first pin (WA is
// shift-invariant), and exponents relative to m+ / m-, so that FP32 keeps the
// digits that matter even where the cells of a net sit close together far
// from the origin.  Nets are grouped by degree at create: groups of G lanes
// (G = 4, 8, 16, 32) handle one net each, looping for degree > G; nets with
// more than 256 pins get a whole block.  Per-pin gradients are written to a
// pin-ordered array; the per-cell sum runs in the cell-gradient kernel in a
// fixed order (no floating-point atomics, so results are deterministic).
#include <cfloat>

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

template <int G>
__global__ void __launch_bounds__(kThreads) k_wa_group(Dev d, int copy0, int cls, int eval,
                                                        const float *gamma_ovr) {
  __shared__ float sm[32];
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  const float g = copy_gamma(d, c, gamma_ovr);
  const float ig = 1.0f / g;
  const float *x = d.x + (size_t)c * d.n_cells;
  const float *y = d.y + (size_t)c * d.n_cells;
  float2 *pg = d.pin_grad + (size_t)c * d.n_pins;
  constexpr int NPB = kThreads / G;
  const int lane = threadIdx.x % G;
  const int e_end = d.cls_begin[cls + 1];
  float hp_acc = 0.f, wl_acc = 0.f;
  for (int base = d.cls_begin[cls] + blockIdx.x * NPB; base < e_end; base += gridDim.x * NPB) {
    const int e = base + threadIdx.x / G;
    const bool valid = e < e_end;
    int p0 = 0, p1 = 0;
    if (valid) {
      p0 = d.net_ptr[e];
      p1 = d.net_ptr[e + 1];
    }
    const float wn = (valid && d.net_w) ? d.net_w[e] : 1.0f;
    // coordinates relative to the net's first pin: (x_j - x_0) + (dx_j - dx_0)
    // rounds relative to the pin spacing, not to the absolute position
    float rx = 0.f, ry = 0.f, rdx = 0.f, rdy = 0.f;
    if (p1 > p0) {
      int cell = d.pin_cell[p0];
      float2 o = d.pin_off[p0];
      rx = x[cell]; ry = y[cell]; rdx = o.x; rdy = o.y;
    }
    // first pin of each lane stays in registers; higher degrees reload
    const int j0 = p0 + lane;
    const bool has0 = j0 < p1;
    float px0 = 0.f, py0 = 0.f;
    if (has0) {
      int cell = d.pin_cell[j0];
      float2 o = d.pin_off[j0];
      px0 = (x[cell] - rx) + (o.x - rdx);
      py0 = (y[cell] - ry) + (o.y - rdy);
    }
    float mxx = has0 ? px0 : -FLT_MAX, mnx = has0 ? px0 : FLT_MAX;
    float mxy = has0 ? py0 : -FLT_MAX, mny = has0 ? py0 : FLT_MAX;
    for (int j = j0 + G; j < p1; j += G) {
      int cell = d.pin_cell[j];
      float2 o = d.pin_off[j];
      float px = (x[cell] - rx) + (o.x - rdx), py = (y[cell] - ry) + (o.y - rdy);
      mxx = fmaxf(mxx, px); mnx = fminf(mnx, px);
      mxy = fmaxf(mxy, py); mny = fminf(mny, py);
    }
    mxx = gmax<G>(mxx); mnx = gmin<G>(mnx);
    mxy = gmax<G>(mxy); mny = gmin<G>(mny);
    float sxp = 0.f, txp = 0.f, sxm = 0.f, txm = 0.f;
    float syp = 0.f, typ = 0.f, sym = 0.f, tym = 0.f;
    float a0x = 0.f, b0x = 0.f, a0y = 0.f, b0y = 0.f;
    if (has0) {
      a0x = expf((px0 - mxx) * ig); b0x = expf((mnx - px0) * ig);
      sxp += a0x; txp += (px0 - mxx) * a0x; sxm += b0x; txm += (px0 - mnx) * b0x;
      a0y = expf((py0 - mxy) * ig); b0y = expf((mny - py0) * ig);
      syp += a0y; typ += (py0 - mxy) * a0y; sym += b0y; tym += (py0 - mny) * b0y;
    }
    for (int j = j0 + G; j < p1; j += G) {
      int cell = d.pin_cell[j];
      float2 o = d.pin_off[j];
      float px = (x[cell] - rx) + (o.x - rdx), py = (y[cell] - ry) + (o.y - rdy);
      float a = expf((px - mxx) * ig), b = expf((mnx - px) * ig);
      sxp += a; txp += (px - mxx) * a; sxm += b; txm += (px - mnx) * b;
      a = expf((py - mxy) * ig); b = expf((mny - py) * ig);
      syp += a; typ += (py - mxy) * a; sym += b; tym += (py - mny) * b;
    }
    sxp = gsum<G>(sxp); txp = gsum<G>(txp); sxm = gsum<G>(sxm); txm = gsum<G>(txm);
    syp = gsum<G>(syp); typ = gsum<G>(typ); sym = gsum<G>(sym); tym = gsum<G>(tym);
    if (p1 > p0) {
      const float rxp = txp / sxp, rxm = txm / sxm, ryp = typ / syp, rym = tym / sym;
      const float isxp = 1.f / sxp, isxm = 1.f / sxm, isyp = 1.f / syp, isym = 1.f / sym;
      if (has0) {
        float gx = a0x * isxp * (1.f + (px0 - mxx - rxp) * ig) - b0x * isxm * (1.f - (px0 - mnx - rxm) * ig);
        float gy = a0y * isyp * (1.f + (py0 - mxy - ryp) * ig) - b0y * isym * (1.f - (py0 - mny - rym) * ig);
        pg[j0] = make_float2(gx * wn, gy * wn);
      }
      for (int j = j0 + G; j < p1; j += G) {
        int cell = d.pin_cell[j];
        float2 o = d.pin_off[j];
        float px = (x[cell] - rx) + (o.x - rdx), py = (y[cell] - ry) + (o.y - rdy);
        float a = expf((px - mxx) * ig), b = expf((mnx - px) * ig);
        float gx = a * isxp * (1.f + (px - mxx - rxp) * ig) - b * isxm * (1.f - (px - mnx - rxm) * ig);
        a = expf((py - mxy) * ig); b = expf((mny - py) * ig);
        float gy = a * isyp * (1.f + (py - mxy - ryp) * ig) - b * isym * (1.f - (py - mny - rym) * ig);
        pg[j] = make_float2(gx * wn, gy * wn);
      }
      if (lane == 0) {
        hp_acc += wn * ((mxx - mnx) + (mxy - mny));
        wl_acc += wn * (((mxx - mnx) + (rxp - rxm)) + ((mxy - mny) + (ryp - rym)));
      }
    }
  }
  float rh = block_sum_f<kThreads>(hp_acc, sm);
  float rw = block_sum_f<kThreads>(wl_acc, sm);
  if (threadIdx.x == 0) {
    size_t base = (size_t)c * S_COUNT * d.nb_red + d.wa_block_base[cls] + blockIdx.x;
    d.part[base + (size_t)S_HPWL * d.nb_red] = rh;
    d.part[base + (size_t)S_WL * d.nb_red] = rw;
  }
}

// Block-wide reductions for the one-block-per-net kernel.
__device__ __forceinline__ float bred_max(float v, float *sm) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = sm[0];
  for (int i = 1; i < kThreads / 32; ++i) r = fmaxf(r, sm[i]);
  return r;
}
__device__ __forceinline__ float bred_min(float v, float *sm) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = sm[0];
  for (int i = 1; i < kThreads / 32; ++i) r = fminf(r, sm[i]);
  return r;
}
__device__ __forceinline__ float bred_sum(float v, float *sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = sm[0];
  for (int i = 1; i < kThreads / 32; ++i) r += sm[i];
  return r;
}

__global__ void __launch_bounds__(kThreads) k_wa_block(Dev d, int copy0, int cls, int eval,
                                                        const float *gamma_ovr) {
  __shared__ float sm[32];
  const int c = copy0 + blockIdx.y;
  if (!eval && d.cs[c].stopped) return;
  const float g = copy_gamma(d, c, gamma_ovr);
  const float ig = 1.0f / g;
  const float *x = d.x + (size_t)c * d.n_cells;
  const float *y = d.y + (size_t)c * d.n_cells;
  float2 *pg = d.pin_grad + (size_t)c * d.n_pins;
  float hp_acc = 0.f, wl_acc = 0.f;
  for (int e = d.cls_begin[cls] + blockIdx.x; e < d.cls_begin[cls + 1]; e += gridDim.x) {
    const int p0 = d.net_ptr[e], p1 = d.net_ptr[e + 1];
    const float wn = d.net_w ? d.net_w[e] : 1.0f;
    const int cell0 = d.pin_cell[p0];
    const float2 o0 = d.pin_off[p0];
    const float rx = x[cell0], ry = y[cell0], rdx = o0.x, rdy = o0.y;
    float mxx = -FLT_MAX, mnx = FLT_MAX, mxy = -FLT_MAX, mny = FLT_MAX;
    for (int j = p0 + threadIdx.x; j < p1; j += kThreads) {
      int cell = d.pin_cell[j];
      float2 o = d.pin_off[j];
      float px = (x[cell] - rx) + (o.x - rdx), py = (y[cell] - ry) + (o.y - rdy);
      mxx = fmaxf(mxx, px); mnx = fminf(mnx, px);
      mxy = fmaxf(mxy, py); mny = fminf(mny, py);
    }
    mxx = bred_max(mxx, sm); mnx = bred_min(mnx, sm);
    mxy = bred_max(mxy, sm); mny = bred_min(mny, sm);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = p0 + threadIdx.x; j < p1; j += kThreads) {
      int cell = d.pin_cell[j];
      float2 o = d.pin_off[j];
      float px = (x[cell] - rx) + (o.x - rdx), py = (y[cell] - ry) + (o.y - rdy);
      float a = expf((px - mxx) * ig), b = expf((mnx - px) * ig);
      s[0] += a; s[1] += (px - mxx) * a; s[2] += b; s[3] += (px - mnx) * b;
      a = expf((py - mxy) * ig); b = expf((mny - py) * ig);
      s[4] += a; s[5] += (py - mxy) * a; s[6] += b; s[7] += (py - mny) * b;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = bred_sum(s[q], sm);
    const float rxp = s[1] / s[0], rxm = s[3] / s[2], ryp = s[5] / s[4], rym = s[7] / s[6];
    for (int j = p0 + threadIdx.x; j < p1; j += kThreads) {
      int cell = d.pin_cell[j];
      float2 o = d.pin_off[j];
      float px = (x[cell] - rx) + (o.x - rdx), py = (y[cell] - ry) + (o.y - rdy);
      float a = expf((px - mxx) * ig), b = expf((mnx - px) * ig);
      float gx = a / s[0] * (1.f + (px - mxx - rxp) * ig) - b / s[2] * (1.f - (px - mnx - rxm) * ig);
      a = expf((py - mxy) * ig); b = expf((mny - py) * ig);
      float gy = a / s[4] * (1.f + (py - mxy - ryp) * ig) - b / s[6] * (1.f - (py - mny - rym) * ig);
      pg[j] = make_float2(gx * wn, gy * wn);
    }
    hp_acc += wn * ((mxx - mnx) + (mxy - mny));
    wl_acc += wn * (((mxx - mnx) + (rxp - rxm)) + ((mxy - mny) + (ryp - rym)));
    __syncthreads();
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
  const float *x = d.x + (size_t)c * d.n_cells;
  const float *y = d.y + (size_t)c * d.n_cells;
  constexpr int NPB = kThreads / G;
  const int lane = threadIdx.x % G;
  double acc = 0.0;
  for (int base = e_begin + blockIdx.x * NPB; base < e_end; base += gridDim.x * NPB) {
    const int e = base + threadIdx.x / G;
    int p0 = 0, p1 = 0;
    if (e < e_end) {
      p0 = d.net_ptr[e];
      p1 = d.net_ptr[e + 1];
    }
    double mxx = -1e300, mnx = 1e300, mxy = -1e300, mny = 1e300;
    for (int j = p0 + lane; j < p1; j += G) {
      int cell = d.pin_cell[j];
      float2 o = d.pin_off[j];
      double px = (double)x[cell] + (double)o.x, py = (double)y[cell] + (double)o.y;
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

void launch_wa(const Dev &d, int copy0, int ncopy, int eval, const float *gamma_ovr,
               cudaStream_t st) {
  for (int cls = 0; cls < d.n_cls; ++cls) {
    int nb = d.wa_blocks[cls];
    if (nb == 0) continue;
    dim3 grid(nb, ncopy);
    switch (cls) {
      case 0: k_wa_group<4><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr); break;
      case 1: k_wa_group<8><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr); break;
      case 2: k_wa_group<16><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr); break;
      case 3: k_wa_group<32><<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr); break;
      default: k_wa_block<<<grid, kThreads, 0, st>>>(d, copy0, cls, eval, gamma_ovr); break;
    }
  }
}

int hpwl64_blocks(const Dev &d) { return 2 * d.cell_blocks; }

void launch_hpwl64(const Dev &d, int copy0, int ncopy, cudaStream_t st) {
  // small nets: 4 lanes each; nets with more than 4 pins: a warp each
  const int split = d.cls_begin[1];
  dim3 grid(d.cell_blocks, ncopy);
  k_hpwl64<4><<<grid, kThreads, 0, st>>>(d, copy0, 0, split, 0);
  k_hpwl64<32><<<grid, kThreads, 0, st>>>(d, copy0, split, d.n_nets, d.cell_blocks);
}

}  // namespace hp
