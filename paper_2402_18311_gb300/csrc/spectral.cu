// Spectral Poisson solve as chains of dense transforms (the ePlace
// electrostatic system the paper cites): with C[u][x] = cos(pi u (x+1/2)/M),
// S[x][u] = sin(pi u (x+1/2)/M) and continuous wavenumbers
// w_u = pi u / (M h_x):
//   a_uv  = c_u c_v / (M N) sum_x sum_y rho_xy C_M[u][x] C_N[v][y]
//   Ex_xy = sum_uv a_uv w_u / (w_u^2 + w_v^2) S_M[x][u] C_N[y][v]
//   Ey_xy = sum_uv a_uv w_v / (w_u^2 + w_v^2) C_M[x][u] S_N[y][v]
//   psi_xy = sum_uv a_uv / (w_u^2 + w_v^2) C_M[x][u] C_N[y][v]    ((u,v) != 0)
// Every step is one GEMM D = A B^T with both operands K-major (row-major,
// K contiguous):
//   G1  T1[v][x]  = sum_y Cn[v][y]  rho[x][y]
//   G2  A^[u][v]  = sum_x Cm[u][x]  T1[v][x]    epilogue: spectral weights -> Bx, By (, Bpsi)
//   G3  T[w][y][u] = sum_v An_w[y][v] B_w[u][v]  An = (C_N^T, S_N, C_N^T) for (x, y, psi)
//   G4  E[w][x][y] = sum_u Am_w[x][u] T[w][y][u] Am = (S_M, C_M^T, C_M^T)
// so no transpose pass is needed between steps.
//
// This file holds the FP32 CUDA-core GEMM (64x64x16 tiles, 4x4 register
// micro-tiles); the tensor-core BF16x3 path lives in spectral_tc.cu.
#include "common.cuh"
#include "internal.cuh"
#include "spectral_tc.cuh"

namespace hp {

struct GemmArgs {
  const float *A[3];
  const float *B;
  long long sBw, sBc;  // stride between 'which' and between copies
  float *D;
  long long sDw, sDc;
  int M, N, K;         // D is M x N, contraction K
  int nwhich, copy0;
  int spectral;        // G2 epilogue
  int with_psi;
  const float *wu, *wv, *cu, *cv;
  const CopyState *cs;
  int eval;
};

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256) k_gemm_nt(GemmArgs g) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int z = blockIdx.z;
  const int which = z % g.nwhich;
  const int c = g.copy0 + z / g.nwhich;
  if (!g.eval && g.cs[c].stopped) return;
  const float *A = g.A[which];
  const float *B = g.B + which * g.sBw + c * g.sBc;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int lr = tid >> 2, lk = (tid & 3) * 4;  // loader: row, k offset
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    float4 av = make_float4(0.f, 0.f, 0.f, 0.f), bv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m0 + lr < g.M) av = *reinterpret_cast<const float4 *>(A + (size_t)(m0 + lr) * g.K + k0 + lk);
    if (n0 + lr < g.N) bv = *reinterpret_cast<const float4 *>(B + (size_t)(n0 + lr) * g.K + k0 + lk);
    As[lk + 0][lr] = av.x; As[lk + 1][lr] = av.y; As[lk + 2][lr] = av.z; As[lk + 3][lr] = av.w;
    Bs[lk + 0][lr] = bv.x; Bs[lk + 1][lr] = bv.y; Bs[lk + 2][lr] = bv.z; Bs[lk + 3][lr] = bv.w;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a4 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      float4 b4 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *D = g.D + which * g.sDw + c * g.sDc;
  const size_t GN = (size_t)g.M * g.N;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      const size_t o = (size_t)m * g.N + n;
      if (!g.spectral) {
        D[o] = acc[i][j];
      } else {
        const float a = acc[i][j] * g.cu[m] * g.cv[n];
        const float wu = g.wu[m], wv = g.wv[n];
        const float den = wu * wu + wv * wv;
        const bool dc = (m == 0 && n == 0);
        const float inv = dc ? 0.f : 1.f / den;
        D[o] = a * wu * inv;
        D[GN + o] = a * wv * inv;
        if (g.with_psi) D[2 * GN + o] = a * inv;
      }
    }
  }
}

static void gemm(const GemmArgs &g, int ncopy, cudaStream_t st) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.nwhich * ncopy);
  k_gemm_nt<<<grid, 256, 0, st>>>(g);
}

void launch_spectral_fp32(const Dev &d, int copy0, int ncopy, int with_psi, int eval,
                          cudaStream_t st) {
  const int M = d.nx, N = d.ny;
  const long long G = d.G;
  GemmArgs g = {};
  g.copy0 = copy0;
  g.cs = d.cs;
  g.eval = eval;
  g.wu = d.wu; g.wv = d.wv; g.cu = d.cu; g.cv = d.cv;
  // G1: T1 = Cn * rho^T   (N x M, K = N)
  g.A[0] = d.Cn;
  g.B = d.rho; g.sBw = 0; g.sBc = G;
  g.D = d.T; g.sDw = 0; g.sDc = 3 * G;
  g.M = N; g.N = M; g.K = N; g.nwhich = 1; g.spectral = 0;
  gemm(g, ncopy, st);
  // G2: A^ = Cm * T1^T   (M x N, K = M), spectral epilogue into SB
  g.A[0] = d.Cm;
  g.B = d.T; g.sBw = 0; g.sBc = 3 * G;
  g.D = d.SB; g.sDw = 0; g.sDc = 3 * G;
  g.M = M; g.N = N; g.K = M; g.spectral = 1; g.with_psi = with_psi;
  gemm(g, ncopy, st);
  // G3: T[w] = An_w * B_w^T   (N x M, K = N)
  g.A[0] = d.CTn; g.A[1] = d.STn; g.A[2] = d.CTn;
  g.B = d.SB; g.sBw = G; g.sBc = 3 * G;
  g.D = d.T; g.sDw = G; g.sDc = 3 * G;
  g.M = N; g.N = M; g.K = N; g.spectral = 0; g.nwhich = with_psi ? 3 : 2;
  gemm(g, ncopy, st);
  // G4: E[w] = Am_w * T[w]^T   (M x N, K = M)
  g.A[0] = d.STm; g.A[1] = d.CTm; g.A[2] = d.CTm;
  g.B = d.T; g.sBw = G; g.sBc = 3 * G;
  g.D = d.E; g.sDw = G; g.sDc = 3 * G;
  g.M = M; g.N = N; g.K = M;
  gemm(g, ncopy, st);
}

// Tensor-core chain (BF16x3): rho_hl -> T_hl[0] -> SB_hl -> T_hl[w] -> E[w].
// Stage 2 writes one coefficient field, B = a / (w_u^2 + w_v^2); stage 3
// reads it for every field w: its y matrix holds S_N with column v scaled by
// w_v, and its x output's columns u are scaled by w_u, which gives the field
// coefficients w_u B and w_v B of the FP32 chain above (psi takes B as is).
//
// Even/odd split (d.bfly; both sides multiples of 256).  With
// c_k(i) = cos(pi k (i + 1/2) / L) and s_k(i) = sin(pi k (i + 1/2) / L),
// c_k(L-1-i) = (-1)^k c_k(i) and s_k(L-1-i) = (-1)^(k+1) s_k(i).  So a
// forward cosine transform needs, for its even frequencies, only the sums
// x_i + x_{L-1-i} and, for its odd ones, only the differences (i < L/2):
// half the contraction.  An inverse transform gives, with E_i and O_i its
// sums over the even and over the odd frequencies (i < L/2),
// x_i = E_i + O_i and x_{L-1-i} = +-(E_i - O_i) (+ for cosines, - for
// sines): half the rows, each contracted over all frequencies.  Frequencies
// are kept in the order 0, 2, 4, ..., 1, 3, 5, ... between the stages, so
// the even and odd halves are the two halves of every contraction:
//   rho' = rho's y-halves (sums, differences)     (density finish)
//   stage 1: T' rows in that order; its epilogue writes the x-halves of T
//            (each CTA holds columns x and nx-1-x)
//   stage 2: forward along x on T', the coefficient field in that order
//   stage 3: inverse along y (rows y < ny/2 and their mirrors)
//   stage 4: inverse along x: the field in natural order
// Every stage does half the tensor-core work of the plain chain.
namespace {

void stage_args(const Dev &d, int stage, int with_psi, TcArgs &g) {
  const int f = d.bfly;
  g.b_koff = g.fold = g.mirror = 0;
  if (stage == 0) {
    // G1: T[0] = Cn rho^T   (ny x nx, K = ny)
    g.M = d.ny; g.N = d.nx; g.K = f ? d.ny / 2 : d.ny; g.nwhich = 1;
    g.b_per_copy = 1; g.b_shared = 0; g.d_per_copy = 3; g.col_scale = nullptr;
    g.epi = TC_EPI_SPLIT; g.Dh = d.T_h; g.Dl = d.T_l;
    g.b_koff = f ? d.ny / 2 : 0;
    g.fold = f;
  } else if (stage == 1) {
    // G2: SB = spectral(Cm T[0]^T)   (nx x ny, K = nx), one field per copy
    g.M = d.nx; g.N = d.ny; g.K = f ? d.nx / 2 : d.nx; g.nwhich = 1;
    g.b_per_copy = 3; g.b_shared = 0; g.d_per_copy = 1; g.col_scale = nullptr;
    g.epi = TC_EPI_SPECTRAL; g.Dh = d.SB_h; g.Dl = d.SB_l;
    g.b_koff = f ? d.nx / 2 : 0;
  } else if (stage == 2) {
    // G3: T[w] = An_w SB^T   (ny x nx, K = ny), the x output scaled by w_u
    g.M = d.ny; g.N = d.nx; g.K = d.ny; g.nwhich = with_psi ? 3 : 2;
    g.b_per_copy = 1; g.b_shared = 1; g.d_per_copy = 3; g.col_scale = f ? d.wu_p : d.wu;
    g.epi = TC_EPI_SPLIT; g.Dh = d.T_h; g.Dl = d.T_l;
    g.mirror = f;
    g.msign[0] = 1.f; g.msign[1] = -1.f; g.msign[2] = 1.f;  // y: cos, sin, cos
  } else {
    // G4: E[w] = Am_w T[w]^T   (nx x ny, K = nx)
    g.M = d.nx; g.N = d.ny; g.K = d.nx; g.nwhich = with_psi ? 3 : 2;
    g.b_per_copy = 3; g.b_shared = 0; g.d_per_copy = 3; g.col_scale = nullptr;
    g.epi = TC_EPI_F32; g.Df = d.E; g.Dh = g.Dl = nullptr;
    g.mirror = f;
    g.msign[0] = -1.f; g.msign[1] = 1.f; g.msign[2] = 1.f;  // x: sin, cos, cos
  }
}

void base_args(const Dev &d, int copy0, int eval, int with_psi, TcArgs &g) {
  g = TcArgs{};
  g.copy0 = copy0;
  g.cs = d.cs;
  g.eval = eval;
  g.err = d.err;
  const bool f = d.bfly != 0;
  g.wu = f ? d.wu_p : d.wu; g.wv = f ? d.wv_p : d.wv;
  g.cu = f ? d.cu_p : d.cu; g.cv = f ? d.cv_p : d.cv;
  g.with_psi = with_psi;
  g.ws = d.tc_ws;
  g.ws_ctr = d.tc_ws_ctr;
}

}  // namespace

void launch_spectral_tc(const Dev &d, int copy0, int ncopy, int with_psi, int eval,
                        cudaStream_t st) {
  const CUtensorMap *mp = static_cast<const CUtensorMap *>(d.tcm);
  TcArgs g;
  base_args(d, copy0, eval, with_psi, g);
  for (int s = 0; s < 4; ++s) {
    stage_args(d, s, with_psi, g);
    // with psi the last two stages have a third field: more tiles than the
    // split-K workspace holds, so one CTA per tile (the same bits)
    const int split = (with_psi && s >= 2) ? 1 : d.tc_split[s];
    launch_tc_gemm(mp + 4 * s, g, ncopy, d.tc_bn[s], split, st);
  }
}

// The first GEMM stage of copy 0 with its producer idle: no tile ever lands,
// so the MMA issuer's and the epilogue's bounded waits give up (about a
// second each) and the kernel raises d.err instead of hanging.
void launch_spectral_tc_stalled(const Dev &d, cudaStream_t st) {
  const CUtensorMap *mp = static_cast<const CUtensorMap *>(d.tcm);
  TcArgs g;
  base_args(d, 0, 1, 0, g);
  g.no_load = 1;
  stage_args(d, 0, 0, g);
  launch_tc_gemm(mp + 0, g, 1, d.tc_bn[0], d.tc_split[0], st);
}

void launch_spectral(const Dev &d, int copy0, int ncopy, int with_psi, int eval,
                     cudaStream_t st) {
  if (d.tc)
    launch_spectral_tc(d, copy0, ncopy, with_psi, eval, st);
  else
    launch_spectral_fp32(d, copy0, ncopy, with_psi, eval, st);
}

}  // namespace hp
