// Tensor-core (tcgen05) GEMM stage of the spectral Poisson solve: interface.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace hp {

struct CopyState;

enum { TC_EPI_F32 = 0, TC_EPI_SPLIT = 1, TC_EPI_SPECTRAL = 2 };

// One batched GEMM D[b] = A[which] B[b]^T, b = copy * per_copy + which.
struct TcArgs {
  int M, N, K;                 // D is M x N per batch; contraction over K
  int nwhich, copy0;
  int b_per_copy, d_per_copy;  // batch slots per copy in B and in D
  int b_shared;                // 1: every `which` reads the copy's one B (batch c * b_per_copy)
  const float *col_scale;      // TC_EPI_SPLIT: the which == 0 output's columns n are scaled
                               // by col_scale[n] (nullptr: none)
  int epi, with_psi;
  float *Df;                   // TC_EPI_F32 output
  __nv_bfloat16 *Dh, *Dl;      // split outputs
  const float *wu, *wv, *cu, *cv;
  const CopyState *cs;
  int eval;
  int *err;                    // set to 1 when a bounded wait gives up
  float *ws;                   // split-K: [tiles][2][128][BN] partial halves
  unsigned int *ws_ctr;        // split-K: arrivals per tile (reset by the second)
  int no_load;                 // 1: the producer issues no copies (failure-path check:
                               // the consumers' bounded waits give up)
  // Even/odd split of a length-L transform (L a multiple of 256; see
  // spectral.cu): with x'_i = x_i + x_{L-1-i} and x''_i = x_i - x_{L-1-i}
  // (i < L/2) the forward cosine transform's even frequencies need only x'
  // and its odd ones only x''; an inverse transform's outputs i and L-1-i
  // share the sums E_i over the even frequencies and O_i over the odd ones.
  int b_koff;                  // forward: K is the half length; output rows m >= M/2 (the odd
                               // frequencies) read B from K offset b_koff (x''), the others
                               // from 0 (x'); 0: off
  int fold;                    // TC_EPI_SPLIT: the CTA's B tile is rows [f BN/2, (f+1) BN/2)
                               // and their mirrors N-1-n (f = tile column), and the epilogue
                               // writes the split pair (x', x'') of its N/2-wide halves
  int mirror;                  // inverse: the grid covers rows m < M/2; the two K halves
                               // (even, odd frequencies) give E and O, row m gets E + O and
                               // row M-1-m gets msign[which] (E - O)
  float msign[3];
};

int tc_smem_bytes(int bn);
int tc_prepare();
void launch_tc_gemm(const CUtensorMap *maps4, const TcArgs &g, int ncopy, int bn, int split,
                    cudaStream_t st);
void launch_split_bf16(const float *src, __nv_bfloat16 *hi, __nv_bfloat16 *lo, size_t n,
                       cudaStream_t st);
// The same for a rows x cols row-major matrix whose column j is first scaled
// by w[j] (one FP32 product per element).
void launch_split_bf16_colscale(const float *src, const float *w, __nv_bfloat16 *hi,
                                __nv_bfloat16 *lo, int rows, int cols, cudaStream_t st);
// 3D bf16 tensor map {K, rows, batch} with a {64, box_rows, 1} box and
// 128-byte swizzle; returns 0 on success.
int make_map_bf16_3d(CUtensorMap *map, const void *base, int K, int rows, int batch, int box_rows);

}  // namespace hp
