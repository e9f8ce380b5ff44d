// Spectral Poisson solve on the 5th-generation tensor cores (tcgen05).
//
// Same chain of four GEMM stages as spectral.cu (D = A B^T, both operands
// K-major), computed as BF16x3: every FP32 operand is split into
// hi = bf16(x) and lo = bf16(x - hi), and
//     D = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// accumulates in FP32 in tensor memory.  The transform matrices are split
// once at create; every data operand is split by the kernel that produces it
// (density finish for rho, the GEMM epilogues for the intermediates), so the
// GEMMs read bf16 pairs straight from global memory.
//
// Kernel layout: one 128 x BN output tile per CTA of 4 warps.  Warp 0 (one
// lane) streams K-blocks of 64 elements of A_hi, A_lo, B_hi, B_lo into a
// 3-stage shared-memory ring with TMA (128-byte swizzle); warp 1 (one lane)
// issues tcgen05.mma (M=128, N=BN, K=16) into TMEM accumulators and frees
// each stage with tcgen05.commit; then all four warps read the accumulators
// with tcgen05.ld and run the fused epilogue (plain FP32 store, bf16 split,
// the spectral weights of the Poisson solve, or the even/odd combinations
// of spectral.cu).  Every wait on an mbarrier gives up after about a second
// of clock cycles and raises an error flag instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.cuh"
#include "spectral_tc.cuh"

namespace hp {

namespace tc {

constexpr int BM = 128, BKE = 64;   // tile rows, bf16 K elements per stage
constexpr int TILE_A = BM * BKE * 2;  // bytes of one A_hi or A_lo stage tile
constexpr long long kWaitCycles = 2000000000ll;  // about one second

template <int BN, int STAGES>
struct Cfg {
  static constexpr int TILE_B = BN * BKE * 2;
  static constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;  // ring, alignment, barriers
  // Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = BN.
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after about kWaitCycles without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart, SM100 descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 columns of this warp's 32 TMEM lanes; tmem_wait() makes them valid.
__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One 32-byte global store (a whole sector); p is 32-byte aligned.
__device__ __forceinline__ void st_v8(void *p, uint4 a, uint4 b) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a.x),
               "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

// The two K halves of 32 accumulator columns from cc: with SPLIT = 1 both
// are this CTA's (TMEM columns cc and BN + cc), with SPLIT = 2 one is this
// CTA's (half ks) and the other the partner's, from the workspace.
template <int BN, int SPLIT>
__device__ __forceinline__ void acc_halves(uint32_t trow, int cc, const float *ws_other, int ks,
                                           float (&h0)[32], float (&h1)[32]) {
  uint32_t r[32];
  if constexpr (SPLIT == 1) {
    // both halves in flight before one wait
    uint32_t r2[32];
    tmem_ld32_nw(trow + (uint32_t)cc, r);
    tmem_ld32_nw(trow + (uint32_t)(BN + cc), r2);
    tmem_wait();
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      h0[i] = __uint_as_float(r[i]);
      h1[i] = __uint_as_float(r2[i]);
    }
  } else {
    tmem_ld32(trow + (uint32_t)cc, r);
    const float4 *src = reinterpret_cast<const float4 *>(ws_other + cc);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 q = __ldcg(src + i);
      const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float own = __uint_as_float(r[4 * i + j]);
        h0[4 * i + j] = ks == 0 ? own : qv[j];
        h1[4 * i + j] = ks == 0 ? qv[j] : own;
      }
    }
  }
}

// Their sum: the tile's 32 output values (addition is commutative, so the
// split and unsplit kernels give the same bits).
template <int BN, int SPLIT>
__device__ __forceinline__ void acc_sum(uint32_t trow, int cc, const float *ws_other, int ks,
                                        float (&v)[32]) {
  float h1[32];
  acc_halves<BN, SPLIT>(trow, cc, ws_other, ks, v, h1);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __fadd_rn(v[i], h1[i]);
}

__device__ __forceinline__ void split_store(__nv_bfloat16 *hi, __nv_bfloat16 *lo, const float *v) {
  // 32 consecutive values -> 32 bf16 hi and 32 bf16 lo (64 bytes each)
  __align__(16) __nv_bfloat16 h[32];
  __align__(16) __nv_bfloat16 l[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    h[i] = __float2bfloat16_rn(v[i]);
    l[i] = __float2bfloat16_rn(v[i] - __bfloat162float(h[i]));
  }
  uint4 *dh = reinterpret_cast<uint4 *>(hi), *dl = reinterpret_cast<uint4 *>(lo);
  const uint4 *sh = reinterpret_cast<const uint4 *>(h), *sl = reinterpret_cast<const uint4 *>(l);
#pragma unroll
  for (int i = 0; i < 4; i += 2) {
    st_v8(dh + i, sh[i], sh[i + 1]);
    st_v8(dl + i, sl[i], sl[i + 1]);
  }
}

// 32 consecutive FP32 outputs at element o of the output (column n of the
// row): stored as they are (TC_EPI_F32) or as a bf16 pair (TC_EPI_SPLIT,
// the which == 0 output scaled by col_scale[n] first).
__device__ __forceinline__ void store_out(const TcArgs &g, int which, size_t o, int n,
                                          float (&v)[32]) {
  if (g.epi == TC_EPI_F32) {
    uint4 *dst = reinterpret_cast<uint4 *>(g.Df + o);
#pragma unroll
    for (int i = 0; i < 8; i += 2)
      st_v8(dst + i,
            make_uint4(__float_as_uint(v[4 * i]), __float_as_uint(v[4 * i + 1]),
                       __float_as_uint(v[4 * i + 2]), __float_as_uint(v[4 * i + 3])),
            make_uint4(__float_as_uint(v[4 * i + 4]), __float_as_uint(v[4 * i + 5]),
                       __float_as_uint(v[4 * i + 6]), __float_as_uint(v[4 * i + 7])));
  } else {
    if (g.col_scale && which == 0) {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = __fmul_rn(v[i], g.col_scale[n + i]);
    }
    split_store(g.Dh + o, g.Dl + o, v);
  }
}

}  // namespace tc

using namespace tc;

// D[z] = A[which] x B[z]^T over one 128 x BN tile; z = copy * nwhich + which.
//
// The contraction is always accumulated as two halves of K, in two TMEM
// accumulators, and the tile is their sum: with SPLIT = 1 one CTA runs both
// halves; with SPLIT = 2 (split-K, for stages with too few tiles to fill the
// SMs) two CTAs run one half each, both publish their half to a workspace,
// and the second to finish adds the other's half to its own and runs the
// epilogue.  Addition is commutative, so every variant gives the same bits.
template <int BN, int STAGES, int SPLIT>
__global__ void __launch_bounds__(128, 1)
    k_umma_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                TcArgs g) {
  extern __shared__ unsigned char smem_raw[];
  const int z = blockIdx.z;
  const int which = z % g.nwhich;
  const int c = g.copy0 + z / g.nwhich;
  if (!g.eval && g.cs[c].stopped) return;
  const int mt = blockIdx.y / SPLIT, ks = blockIdx.y % SPLIT;
  const int m0 = mt * BM, n0 = blockIdx.x * BN;
  const int bz = c * g.b_per_copy + (g.b_shared ? 0 : which);  // batch index of B
  const int dz = c * g.d_per_copy + which;  // batch index of D
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int TCOLS = SPLIT == 1 ? 2 * BN : BN;  // TMEM columns: one accumulator per half here

  using C = Cfg<BN, STAGES>;
  constexpr int TILE_B = C::TILE_B, STAGE_BYTES = C::STAGE_BYTES;
  uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
  unsigned char *tiles = reinterpret_cast<unsigned char *>(base);
  uint64_t *full = reinterpret_cast<uint64_t *>(tiles + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *done = empty + STAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
  int *last_flag = abort_flag + 1;
  __shared__ float s_wv[BN], s_cv[BN];  // spectral epilogue: the tile's column weights
  if (g.epi == TC_EPI_SPECTRAL) {
    for (int i = threadIdx.x; i < BN; i += blockDim.x) {
      s_wv[i] = g.wv[n0 + i];
      s_cv[i] = g.cv[n0 + i];
    }
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *last_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int nhalf = g.K / BKE / 2;  // K-blocks per half (K is a multiple of 128)
  const int kb0 = ks * nhalf;       // this CTA's first K-block
  const int nk = SPLIT == 1 ? 2 * nhalf : nhalf;
  const bool fold = g.fold != 0, mirror = g.mirror != 0;
  // forward even/odd split: the odd-frequency rows read the second half of B
  const int kxb = (g.b_koff && m0 >= g.M / 2) ? g.b_koff : 0;

  // Programmatic launch: everything up to here, and the loads of the
  // constant operand A into the first ring stages, overlaps the end of the
  // kernel before (which lets this one launch once its epilogue starts);
  // B and every output wait for it to complete.  The copy's stopped flag
  // and the tables read above are written by earlier kernels only.
  const int npre = g.no_load ? 0 : (nk < STAGES ? nk : STAGES);
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < npre; ++kb) {
      unsigned char *st = tiles + kb * STAGE_BYTES;
      const int kx = (kb0 + kb) * BKE;
      mbar_expect_tx(&full[kb], STAGE_BYTES);
      tma_load_3d(st, &mAh, &full[kb], kx, m0, which);
      tma_load_3d(st + TILE_A, &mAl, &full[kb], kx, m0, which);
    }
  }
  pdl_wait();
  if (warp == 0 && lane == 0) {
    // producer
    int issued = 0;
    for (int kb = 0; kb < (g.no_load ? 0 : nk); ++kb) {
      const int s = kb % STAGES;
      const int round = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], (round - 1) & 1)) {
        *abort_flag = 1;
        break;
      }
      if (*(volatile int *)abort_flag) break;
      unsigned char *st = tiles + s * STAGE_BYTES;
      const int kx = (kb0 + kb) * BKE;
      if (kb >= npre) {
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_3d(st, &mAh, &full[s], kx, m0, which);
        tma_load_3d(st + TILE_A, &mAl, &full[s], kx, m0, which);
      }
      if (fold) {
        // two half-height boxes (the map's box is BN/2 rows): rows from
        // f BN/2 and their mirrors, stacked in the order of a full box
        constexpr int HB = BN / 2;
        const int r0 = blockIdx.x * HB, r1 = g.N - (blockIdx.x + 1) * HB;
        tma_load_3d(st + 2 * TILE_A, &mBh, &full[s], kxb + kx, r0, bz);
        tma_load_3d(st + 2 * TILE_A + HB * BKE * 2, &mBh, &full[s], kxb + kx, r1, bz);
        tma_load_3d(st + 2 * TILE_A + TILE_B, &mBl, &full[s], kxb + kx, r0, bz);
        tma_load_3d(st + 2 * TILE_A + TILE_B + HB * BKE * 2, &mBl, &full[s], kxb + kx, r1, bz);
      } else {
        tma_load_3d(st + 2 * TILE_A, &mBh, &full[s], kxb + kx, n0, bz);
        tma_load_3d(st + 2 * TILE_A + TILE_B, &mBl, &full[s], kxb + kx, n0, bz);
      }
      issued = kb + 1;
    }
    // make sure no copy is still landing in shared memory when the CTA ends
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb) {
      if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) {
        *abort_flag = 1;
        break;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: the first nhalf K-blocks into columns [0, BN), the rest
    // (SPLIT = 1) into [BN, 2 BN), each half starting from zero
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
        ok = false;
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = smem_u32(tiles + s * STAGE_BYTES);
      const uint32_t ah = st, al = st + TILE_A, bh = st + 2 * TILE_A, bl = st + 2 * TILE_A + TILE_B;
      const int h = kb >= nhalf ? 1 : 0;
      const uint32_t acc_t = tmem + (uint32_t)(h * BN);
      const int kin = kb - h * nhalf;
#pragma unroll
      for (int k = 0; k < BKE / 16; ++k) {
        const uint32_t off = k * 32;  // 16 bf16 = 32 bytes along K inside the swizzle atom
        const uint32_t acc0 = (kin > 0 || k > 0) ? 1u : 0u;
        umma_bf16(acc_t, sw128_desc(ah + off), sw128_desc(bh + off), C::IDESC, acc0);
        umma_bf16(acc_t, sw128_desc(ah + off), sw128_desc(bl + off), C::IDESC, 1u);
        umma_bf16(acc_t, sw128_desc(al + off), sw128_desc(bh + off), C::IDESC, 1u);
      }
      umma_commit(&empty[s]);
    }
    if (ok) umma_commit(done);
  }
  __syncwarp();

  // epilogue: TMEM lanes 32*warp .. +31 hold rows m0 + 32*warp + lane
  // the tcgen05.ld below is warp-collective: decide per warp
  const bool have = __all_sync(0xffffffffu, mbar_wait(done, 0)) != 0;
  asm volatile("griddepcontrol.launch_dependents;");  // the next kernel may launch
  if (!have) *abort_flag = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  const int m = m0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  float *ws_row = nullptr, *ws_other = nullptr;
  bool run = have;
#ifdef PLACE_DEBUG_BOUNDS
  // the output rows and columns of this warp (run stays warp-uniform: the
  // TMEM loads below are warp-collective)
  run = run && __all_sync(0xffffffffu, HP_IN(g.err, m, g.M, BS_TILE_ROW) &&
                                           HP_IN(g.err, n0 + BN - 1, g.N, BS_TILE_ROW));
#endif
  if constexpr (SPLIT == 2) {
    // publish this half, then the second of the pair to arrive finishes
    const int tile = (z * (int)gridDim.y / SPLIT + mt) * (int)gridDim.x + blockIdx.x;
    ws_row = g.ws + ((size_t)(tile * 2 + ks) * BM + warp * 32 + lane) * BN;
    ws_other = g.ws + ((size_t)(tile * 2 + (ks ^ 1)) * BM + warp * 32 + lane) * BN;
    if (have) {
#pragma unroll 1
      for (int cc = 0; cc < BN; cc += 32) {
        uint32_t r[32];
        tmem_ld32(trow + (uint32_t)cc, r);
        uint4 *dst = reinterpret_cast<uint4 *>(ws_row + cc);
#pragma unroll
        for (int i = 0; i < 8; i += 2)
          st_v8(dst + i, make_uint4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]),
                make_uint4(r[4 * i + 4], r[4 * i + 5], r[4 * i + 6], r[4 * i + 7]));
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int prev = atomicAdd(g.ws_ctr + tile, 1u);
      *last_flag = prev == 1u ? 1 : 0;
      if (prev == 1u) g.ws_ctr[tile] = 0u;  // both halves are in: ready for the next launch
    }
    __syncthreads();
    run = have && *(volatile int *)last_flag != 0;
    if (run) __threadfence();
  }
  if (run && fold) {
    // forward even/odd split of the next stage's contraction: column j
    // (n = f BN/2 + j) pairs with column BN-1-j (its mirror N-1-n)
#pragma unroll 1
    for (int cc = 0; cc < BN / 2; cc += 32) {
      float va[32], vb[32], vd[32];
      acc_sum<BN, SPLIT>(trow, cc, ws_other, ks, va);
      acc_sum<BN, SPLIT>(trow, BN - 32 - cc, ws_other, ks, vb);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float b = vb[31 - i];
        vd[i] = __fsub_rn(va[i], b);
        va[i] = __fadd_rn(va[i], b);
      }
      const size_t o = (size_t)dz * g.M * g.N + (size_t)m * g.N + blockIdx.x * (BN / 2) + cc;
      split_store(g.Dh + o, g.Dl + o, va);
      split_store(g.Dh + o + g.N / 2, g.Dl + o + g.N / 2, vd);
    }
  } else if (run && mirror) {
    // inverse even/odd split: E (first K half) and O (second K half) give
    // rows m and M-1-m
    const float sg = g.msign[which];
    const size_t o0 = (size_t)dz * g.M * g.N + (size_t)m * g.N + n0;
    const size_t o1 = (size_t)dz * g.M * g.N + (size_t)(g.M - 1 - m) * g.N + n0;
#pragma unroll 1
    for (int cc = 0; cc < BN; cc += 32) {
      float ve[32], vo[32];
      acc_halves<BN, SPLIT>(trow, cc, ws_other, ks, ve, vo);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float e = ve[i], od = vo[i];
        ve[i] = __fadd_rn(e, od);
        vo[i] = sg > 0.f ? __fsub_rn(e, od) : __fsub_rn(od, e);
      }
      store_out(g, which, o0 + cc, n0 + cc, ve);
      store_out(g, which, o1 + cc, n0 + cc, vo);
    }
  } else if (run) {
#pragma unroll 1
    for (int cc = 0; cc < BN; cc += 32) {
      float v[32];
      acc_sum<BN, SPLIT>(trow, cc, ws_other, ks, v);
      const int n = n0 + cc;
      const size_t o = (size_t)dz * g.M * g.N + (size_t)m * g.N + n;
      if (g.epi != TC_EPI_SPECTRAL) {
        store_out(g, which, o, n, v);
      } else {
        // spectral weights: a_uv = acc c_u c_v/(M N) and the one field
        // B_uv = a_uv / (w_u^2 + w_v^2), the potential's coefficients; the
        // field coefficients w_u B and w_v B are formed by the next stage (w_u
        // scales its x output's columns, w_v its y matrix's columns)
        const size_t G = (size_t)g.M * g.N;
        const size_t ob = (size_t)c * g.d_per_copy * G + (size_t)m * g.N + n;
        const float cu = g.cu[m], wu = g.wu[m], wu2 = wu * wu;
        float bp[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float wv = s_wv[cc + i];
          // fast reciprocal (2 ulp), far below the BF16x3 error of the solve
          const float inv = (m == 0 && n + i == 0) ? 0.f : __fdividef(1.f, fmaf(wv, wv, wu2));
          bp[i] = v[i] * cu * s_cv[cc + i] * inv;
        }
        split_store(g.Dh + ob, g.Dl + ob, bp);
      }
    }
  }
  if (threadIdx.x == 0 && *(volatile int *)abort_flag) atomicExch(g.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

int tc_smem_bytes(int bn) {
  return bn == 64 ? Cfg<64, 2>::SMEM_BYTES : Cfg<128, 3>::SMEM_BYTES;
}

// bn = 128: 3-stage ring, one CTA per SM; bn = 64: 2-stage ring, two CTAs
// per SM (twice the tiles for grids that would leave SMs idle).  split = 2
// (bn = 128 only): two CTAs per tile, one half of K each.
void launch_tc_gemm(const CUtensorMap *maps4, const TcArgs &g, int ncopy, int bn, int split,
                    cudaStream_t st) {
  // with mirror the grid covers the first half of the rows
  const int mrows = g.mirror ? g.M / 2 : g.M;
  dim3 grid(g.N / bn, (mrows / BM) * (split == 2 ? 2 : 1), g.nwhich * ncopy);
  if (bn == 64)
    launch_pdl(k_umma_gemm<64, 2, 1>, grid, dim3(128), Cfg<64, 2>::SMEM_BYTES, st, maps4[0],
               maps4[1], maps4[2], maps4[3], g);
  else if (split == 2)
    launch_pdl(k_umma_gemm<128, 3, 2>, grid, dim3(128), Cfg<128, 3>::SMEM_BYTES, st, maps4[0],
               maps4[1], maps4[2], maps4[3], g);
  else
    launch_pdl(k_umma_gemm<128, 3, 1>, grid, dim3(128), Cfg<128, 3>::SMEM_BYTES, st, maps4[0],
               maps4[1], maps4[2], maps4[3], g);
}

int tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_umma_gemm<128, 3, 1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg<128, 3>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_umma_gemm<128, 3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg<128, 3>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_umma_gemm<64, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg<64, 2>::SMEM_BYTES);
  return e == cudaSuccess ? 0 : -1;
}

// FP32 -> (bf16 hi, bf16 lo) for the static transform matrices.
__global__ void k_split_bf16_colscale(const float *src, const float *w, __nv_bfloat16 *hi,
                                      __nv_bfloat16 *lo, int rows, int cols) {
  const size_t n = (size_t)rows * cols;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = __fmul_rn(src[i], w[i % cols]);
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}
void launch_split_bf16_colscale(const float *src, const float *w, __nv_bfloat16 *hi,
                                __nv_bfloat16 *lo, int rows, int cols, cudaStream_t st) {
  size_t b = ((size_t)rows * cols + 255) / 256;
  int blocks = (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
  k_split_bf16_colscale<<<blocks, 256, 0, st>>>(src, w, hi, lo, rows, cols);
}

__global__ void k_split_bf16(const float *src, __nv_bfloat16 *hi, __nv_bfloat16 *lo, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = src[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

void launch_split_bf16(const float *src, __nv_bfloat16 *hi, __nv_bfloat16 *lo, size_t n,
                       cudaStream_t st) {
  size_t b = (n + 255) / 256;
  int blocks = (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
  k_split_bf16<<<blocks, 256, 0, st>>>(src, hi, lo, n);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int make_map_bf16_3d(CUtensorMap *map, const void *base, int K, int rows, int batch, int box_rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return -1;
    fn = (EncodeTiledFn)p;
  }
  if (((uintptr_t)base & 15) || K % BKE || rows % box_rows) return -2;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)K * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)BKE, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

}  // namespace hp
