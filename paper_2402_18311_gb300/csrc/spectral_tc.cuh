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
