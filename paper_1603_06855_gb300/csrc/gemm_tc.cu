// Split-BF16 tensor-core application of the condensed operator for the mixed form.
//
// Complex N x N operators (the two inverse compliance blocks and the density block) act on
// complex vectors through their real embedding: row 2p+r, column 2q+r' holds
// [[Re, -Im], [Im, Re]] of entry (p, q), so a complex column stored as interleaved
// (re, im) pairs is a real column of length 2N and the product comes out interleaved.
// Both operands are split into three bf16 slices, x = x_hi + x_mid + x_lo (about 24
// significant bits, i.e. FP32 precision), and the product is accumulated in FP32 from the
// six slice products whose order is at most 2^-16: hh, hm, mh, hl, mm, lh.  Sixteen bits
// per operand are not enough on high-contrast cells: the high-wave-number rows of the
// stress product come out of strongly cancelling sums and stall the block iteration near
// a 1e-3 residual.
//
// GEMM kernel (sm_103a): C[col][row] = sum_k A[row][k] B[col][k], both operands K-major
// bf16 in global memory, loaded by TMA (128-byte swizzle) into a 2-stage shared-memory
// ring; one thread issues tcgen05.mma (kind::f16, M = 128, N = 128, K = 16) into an FP32
// accumulator in tensor memory (two halves, alternating by tile); four epilogue warps read it
// back with tcgen05.ld and store FP32.  Warp 0 produces, warp 1 issues MMAs, warps 2-5 drain;
// the kernel is persistent, one CTA per SM walking the output tiles.  Every mbarrier wait is
// bounded: on expiry the kernel records PC_ETIMEOUT in the status word and stops waiting.
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>
#include "gemm_tc.h"
#include "tc_ptx.cuh"

namespace {
using namespace tcx;

constexpr int TC_BM = 128;
constexpr int TC_BN = 128;
constexpr int TC_BK = 64;        // bf16 elements per 128-byte swizzle row
constexpr int TC_STAGES = 2;
constexpr int A_TILE = TC_BM * TC_BK * 2;   // 16 KB
constexpr int B_TILE = TC_BN * TC_BK * 2;   // 32 KB
constexpr int SLICES = 3;
constexpr int STAGE_BYTES = SLICES * (A_TILE + B_TILE);
constexpr int SMEM_BYTES = TC_STAGES * STAGE_BYTES + 1024 /* barriers */ + 1024 /* alignment */;
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major, M = 128, N = TC_BN.
__host__ __device__ constexpr uint32_t idesc_bf16() { return idesc_bf16_n(TC_BN); }

// Persistent: the producer lane claims output tiles from a counter in global memory (M-fastest,
// so CTAs working at the same time share the B column tile in L2) and hands each tile index to
// the MMA lane and the epilogue warps through a 4-deep ring in shared memory; an index >= tiles
// ends all three.  CTAs that start late, behind another stream's kernel on their SM, claim fewer
// tiles instead of holding the launch up.  The last CTA to finish resets the counter for the
// next launch on the same stream.  The stage ring runs on across tiles, and the accumulator
// alternates between two 128-column halves of tensor memory, so the epilogue warps drain tile i
// while the MMAs of tile i + 1 run.
// The GEMMs of one launch: up to three segments, each an operator (A maps) times a range of
// right-hand-side columns (B maps) into its own output; the tiles of segment g are tile0[g] ..
// tile0[g] + mtiles * ntiles[g] - 1, M-fastest.
struct TcSeg {
  int which, bset;         // operator index (A maps), right-hand-side set (B maps)
  int col_base, ncols;     // columns of the right-hand sides (and of the output)
  int tile0, ntiles;       // first tile of the segment, column tiles
  float* C;                // output, column col_base + j at C + (col_base + j) * ldc
};
struct TcGemmParams {
  CUtensorMap A[3][3];     // [operator][slice hi, mid, lo]
  CUtensorMap B[2][3];     // [right-hand-side set][slice]
  TcSeg seg[3];
  int nseg, num_kb, m_valid, mtiles, tiles;
  long long ldc;
  int* tile_ctr;
  int* status;
};
__device__ __forceinline__ int tc_segment(const TcGemmParams& P, int t) {
  int g = 0;
  while (g + 1 < P.nseg && t >= P.seg[g + 1].tile0) ++g;
  return g;
}

__global__ __launch_bounds__(192, 1) void k_tc_gemm(const __grid_constant__ TcGemmParams P) {
  const int num_kb = P.num_kb, m_valid = P.m_valid, mtiles = P.mtiles;
  const long long ldc = P.ldc;
  int* const tile_ctr = P.tile_ctr;
  int* const status = P.status;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t bars = base + TC_STAGES * STAGE_BYTES;
  // barriers: full[s] +8s, empty[s] +64+8s, tfull[b] +128+8b, tempty[b] +160+8b, done +192; tmem slot +256;
  // tile ring: idfull[j] +320+8j, idempty[j] +352+8j, tile index j at +384+4j
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + TC_STAGES * STAGE_BYTES + 256);
  volatile int* tile_id = reinterpret_cast<volatile int*>(gbase + TC_STAGES * STAGE_BYTES + 384);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = P.tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(bars + 8 * s, 1);
      mbar_init(bars + 64 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bars + 128 + 8 * b, 1);
      mbar_init(bars + 160 + 8 * b, 128);
    }
    mbar_init(bars + 192, 1);
    for (int j = 0; j < 4; ++j) {
      mbar_init(bars + 320 + 8 * j, 1);
      mbar_init(bars + 352 + 8 * j, 5);  // the MMA lane and the four epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * TC_BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;  // stage counter across tiles
      bool ok = true;
      for (int tl = 0; ok; ++tl) {
        const int slot = tl & 3;
        if (!(ok = mbar_wait(bars + 352 + 8 * slot, ((uint32_t)(tl >> 2) & 1u) ^ 1u, status))) break;
        const int t = atomicAdd(tile_ctr, 1);
        tile_id[slot] = t;
        mbar_arrive(bars + 320 + 8 * slot);
        if (t >= tiles) break;
        const TcSeg& sg = P.seg[tc_segment(P, t)];
        const int lt = t - sg.tile0;
        const int m0 = (lt % mtiles) * TC_BM, n0 = sg.col_base + (lt / mtiles) * TC_BN;
        const CUtensorMap* Am = P.A[sg.which];
        const CUtensorMap* Bm = P.B[sg.bset];
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = (int)(it % TC_STAGES);
          const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
          if (!(ok = mbar_wait(bars + 64 + 8 * s, ph ^ 1u, status))) break;
          const uint32_t st = base + s * STAGE_BYTES;
          mbar_expect_tx(bars + 8 * s, STAGE_BYTES);
          tma_load_2d(st, &Am[0], bars + 8 * s, kb * TC_BK, m0);
          tma_load_2d(st + A_TILE, &Am[1], bars + 8 * s, kb * TC_BK, m0);
          tma_load_2d(st + 2 * A_TILE, &Am[2], bars + 8 * s, kb * TC_BK, m0);
          tma_load_2d(st + 3 * A_TILE, &Bm[0], bars + 8 * s, kb * TC_BK, n0);
          tma_load_2d(st + 3 * A_TILE + B_TILE, &Bm[1], bars + 8 * s, kb * TC_BK, n0);
          tma_load_2d(st + 3 * A_TILE + 2 * B_TILE, &Bm[2], bars + 8 * s, kb * TC_BK, n0);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16();
      long long it = 0;
      bool ok = true;
      for (int tl = 0; ok; ++tl) {  // tl: local tile index
        const int slot = tl & 3;
        if (!(ok = mbar_wait(bars + 320 + 8 * slot, (uint32_t)(tl >> 2) & 1u, status))) break;
        const int t = tile_id[slot];
        mbar_arrive(bars + 352 + 8 * slot);
        if (t >= tiles) break;
        const int b = tl & 1;
        // accumulator half b must have been drained (its use tl / 2 - 1)
        if (!(ok = mbar_wait(bars + 160 + 8 * b, ((uint32_t)(tl >> 1) & 1u) ^ 1u, status))) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * TC_BN);
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = (int)(it % TC_STAGES);
          const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
          if (!(ok = mbar_wait(bars + 8 * s, ph, status))) break;
          tc_fence_after();
          const uint32_t st = base + s * STAGE_BYTES;
          const uint64_t ah = sw128_desc(st), am = sw128_desc(st + A_TILE), al = sw128_desc(st + 2 * A_TILE);
          const uint64_t bh = sw128_desc(st + 3 * A_TILE), bm = sw128_desc(st + 3 * A_TILE + B_TILE);
          const uint64_t bl = sw128_desc(st + 3 * A_TILE + 2 * B_TILE);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            const uint64_t off = (uint64_t)((kk * 32) >> 4);  // 16 bf16 = 32 bytes along K
            mma_bf16(d, ah + off, bh + off, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, ah + off, bm + off, idesc, 1u);
            mma_bf16(d, am + off, bh + off, idesc, 1u);
            mma_bf16(d, ah + off, bl + off, idesc, 1u);
            mma_bf16(d, am + off, bm + off, idesc, 1u);
            mma_bf16(d, al + off, bh + off, idesc, 1u);
          }
          mma_commit(bars + 64 + 8 * s);  // stage free once these MMAs have read it
        }
        if (ok) mma_commit(bars + 128 + 8 * b);  // accumulator half b complete
      }
      mma_commit(bars + 192);
      mbar_wait(bars + 192, 0u, status);  // every MMA of this CTA has completed
    }
  } else {
    // epilogue warps 2..5: lane quadrant (warp % 4) of the accumulator
    const int quad = warp & 3;
    for (int tl = 0;; ++tl) {
      const int slot = tl & 3;
      if (!__all_sync(0xffffffffu, mbar_wait(bars + 320 + 8 * slot, (uint32_t)(tl >> 2) & 1u, status))) break;
      const int t = tile_id[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + 352 + 8 * slot);
      if (t >= tiles) break;
      const int b = tl & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(bars + 128 + 8 * b, (uint32_t)(tl >> 1) & 1u, status));
      tc_fence_after();
      const TcSeg& sg = P.seg[tc_segment(P, t)];
      const int lt = t - sg.tile0;
      const int row = (lt % mtiles) * TC_BM + quad * 32 + lane;
      const int n0 = (lt / mtiles) * TC_BN;
      const int col_base = sg.col_base, ncols = sg.ncols;
      float* const C = sg.C;
#pragma unroll 1
      for (int c = 0; c < TC_BN / 16; ++c) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * TC_BN + c * 16), v);
        if (!ok || row >= m_valid) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c * 16 + j;
          if (col < ncols) C[(long long)(col_base + col) * ldc + row] = v[j];
        }
      }
      tc_fence_before();
      mbar_arrive(bars + 160 + 8 * b);
      if (!ok) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * TC_BN))
                 : "memory");
  }
  if (threadIdx.x == 0) {  // every claim of this CTA is done; the last CTA resets the counter
    __threadfence();
    if (atomicAdd(tile_ctr + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(tile_ctr, 0);
      atomicExch(tile_ctr + 1, 0);
    }
  }
}

// ---------------------------------------------------------------------------
// Operand preparation.
// Real embedding of a complex N x N operator (SI, times scale) into [Mp][Kp] hi / mid / lo.
__global__ void k_tc_embed(const double2* __restrict__ W, int N, double scale, int Mp, int Kp,
                           __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ mid,
                           __nv_bfloat16* __restrict__ lo) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)Mp * Kp) return;
  int row = (int)(t / Kp), col = (int)(t % Kp);
  double v = 0.0;
  if (row < 2 * N && col < 2 * N) {
    int p = row >> 1, r = row & 1, q = col >> 1, rp = col & 1;
    double2 w = W[(long long)p * N + q];
    double x = (r == rp) ? w.x : (r == 0 ? -w.y : w.y);
    v = x * scale;
  }
  __nv_bfloat16 h = __double2bfloat16(v);
  double r1 = v - (double)__bfloat162float(h);
  __nv_bfloat16 mm = __double2bfloat16(r1);
  double r2 = r1 - (double)__bfloat162float(mm);
  hi[t] = h;
  mid[t] = mm;
  lo[t] = __double2bfloat16(r2);
}

#define RS2 0.70710678118654752440f
#define RS3 0.57735026918962576451f
#define RS6 0.40824829046386301637f

// Strain stacks of X (six per vector) and the three displacement components, written as
// split bf16 K-major columns: E col = s * nvec + vec, X col = vec * 3 + c; K index 2q + {re, im}.
// Slice t of E sits at E + t * es, of X at X + t * xs.
// The three bf16 slices of (v.x, v.y) stored as pairs at p, p + ss, p + 2 ss (p 4-byte aligned).
__device__ __forceinline__ void split3_store2(float2 v, __nv_bfloat16* p, long long ss) {
  __nv_bfloat16 h0, m0, l0, h1, m1, l1;
  split3_bf16(v.x, h0, m0, l0);
  split3_bf16(v.y, h1, m1, l1);
  *reinterpret_cast<__nv_bfloat162*>(p) = __halves2bfloat162(h0, h1);
  *reinterpret_cast<__nv_bfloat162*>(p + ss) = __halves2bfloat162(m0, m1);
  *reinterpret_cast<__nv_bfloat162*>(p + 2 * ss) = __halves2bfloat162(l0, l1);
}

__global__ void k_tc_split_strain(const float2* __restrict__ X, int nvec, int m, Geom g, const double* __restrict__ Q,
                                  const float4* __restrict__ Kf, int Kp, __nv_bfloat16* __restrict__ E, long long es,
                                  __nv_bfloat16* __restrict__ Xs, long long xs) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int N = g.N;
  const int Kh = Kp / 2;  // complex slots per column (>= N)
  if (t >= (long long)nvec * Kh) return;
  int vec = (int)(t / Kh), q = (int)(t % Kh);
  float2 u0 = make_float2(0.f, 0.f), u1 = u0, u2 = u0;
  float k0 = 0.f, k1 = 0.f, k2 = 0.f;
  if (q < N) {
    const float2* x = X + (long long)vec * 3 * N;
    u0 = x[q]; u1 = x[N + q]; u2 = x[2 * N + q];
    const int k = vec / m;
    if (Kf) {  // the k-set's FP32 wavevectors
      const float4 kk = Kf[(long long)k * N + q];
      k0 = kk.x; k1 = kk.y; k2 = kk.z;
    } else {
      int M2 = 2 * g.M + 1;
      double a0 = Q[3 * k] + (double)(q / (M2 * M2) - g.M);
      double a1 = Q[3 * k + 1] + (double)((q / M2) % M2 - g.M);
      double a2 = Q[3 * k + 2] + (double)(q % M2 - g.M);
      k0 = (float)(g.T[0] * a0 + g.T[1] * a1 + g.T[2] * a2);
      k1 = (float)(g.T[3] * a0 + g.T[4] * a1 + g.T[5] * a2);
      k2 = (float)(g.T[6] * a0 + g.T[7] * a1 + g.T[8] * a2);
    }
  }
  float2 e[6];
  e[0] = make_float2((k0 * u0.x + k1 * u1.x + k2 * u2.x) * RS3, (k0 * u0.y + k1 * u1.y + k2 * u2.y) * RS3);
  e[1] = make_float2((k0 * u0.x - k1 * u1.x) * RS2, (k0 * u0.y - k1 * u1.y) * RS2);
  e[2] = make_float2((k0 * u0.x + k1 * u1.x - 2.f * k2 * u2.x) * RS6, (k0 * u0.y + k1 * u1.y - 2.f * k2 * u2.y) * RS6);
  e[3] = make_float2((k1 * u2.x + k2 * u1.x) * RS2, (k1 * u2.y + k2 * u1.y) * RS2);
  e[4] = make_float2((k0 * u2.x + k2 * u0.x) * RS2, (k0 * u2.y + k2 * u0.y) * RS2);
  e[5] = make_float2((k0 * u1.x + k1 * u0.x) * RS2, (k0 * u1.y + k1 * u0.y) * RS2);
  // (re, im) slices side by side: one 4-byte store per slice (Kp and the slice strides are even)
  for (int s = 0; s < 6; ++s) split3_store2(e[s], E + ((long long)s * nvec + vec) * Kp + 2 * q, es);
  const float2 uu[3] = {u0, u1, u2};
  for (int c = 0; c < 3; ++c) split3_store2(uu[c], Xs + ((long long)vec * 3 + c) * Kp + 2 * q, xs);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  }
  return fn;
}

// 2-D K-major bf16 tensor map: rows x Kp, box TC_BK x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, void* ptr, long long rows, int Kp, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

struct TcPlan {
  int N, nvec_max, Mp, Kp;
  __nv_bfloat16* Ahi[3];  // W1, W2, T_rho (embedded, scaled)
  __nv_bfloat16* Amid[3];
  __nv_bfloat16* Alo[3];
  __nv_bfloat16 *E, *X;   // three slices each: slice t at + t * (rows * Kp)
  float2* S;              // FP32 stress stacks [6][nvec][N]
  CUtensorMap mA_hi[3], mA_mid[3], mA_lo[3], mE[3], mX[3];
  int* status;
  int* tile_ctr;          // tile counter of k_tc_gemm and its finished-CTA count (zero between launches)
  bool ok;
  bool owns_ops;          // false: the operator slices belong to another plan
};

TcPlan* tc_plan_create(int N, int nvec, int* status) {
  TcPlan* p = new TcPlan();  // value-initialised: every pointer starts null
  p->N = N;
  p->nvec_max = nvec;
  p->Mp = ((2 * N + TC_BM - 1) / TC_BM) * TC_BM;
  p->Kp = ((2 * N + TC_BK - 1) / TC_BK) * TC_BK;
  p->status = status;
  p->ok = false;
  p->owns_ops = true;
  size_t asz = (size_t)p->Mp * p->Kp;
  bool good = true;
  for (int i = 0; i < 3; ++i) {
    good &= cudaMalloc(&p->Ahi[i], asz * 2) == cudaSuccess;
    good &= cudaMalloc(&p->Amid[i], asz * 2) == cudaSuccess;
    good &= cudaMalloc(&p->Alo[i], asz * 2) == cudaSuccess;
  }
  size_t esz = (size_t)6 * nvec * p->Kp, xsz = (size_t)3 * nvec * p->Kp;
  good &= cudaMalloc(&p->E, 3 * esz * 2) == cudaSuccess;
  good &= cudaMalloc(&p->X, 3 * xsz * 2) == cudaSuccess;
  good &= cudaMalloc(&p->S, (size_t)6 * nvec * N * sizeof(float2)) == cudaSuccess;
  good &= cudaMalloc(&p->tile_ctr, 2 * sizeof(int)) == cudaSuccess && cudaMemset(p->tile_ctr, 0, 2 * sizeof(int)) == cudaSuccess;
  if (!good) {
    cudaGetLastError();
    tc_plan_destroy(p);
    return nullptr;
  }
  good = true;
  for (int i = 0; i < 3; ++i) {
    good &= make_map(&p->mA_hi[i], p->Ahi[i], p->Mp, p->Kp, TC_BM);
    good &= make_map(&p->mA_mid[i], p->Amid[i], p->Mp, p->Kp, TC_BM);
    good &= make_map(&p->mA_lo[i], p->Alo[i], p->Mp, p->Kp, TC_BM);
  }
  for (int t = 0; t < 3; ++t) {
    good &= make_map(&p->mE[t], p->E + t * esz, (long long)6 * nvec, p->Kp, TC_BN);
    good &= make_map(&p->mX[t], p->X + t * xsz, (long long)3 * nvec, p->Kp, TC_BN);
  }
  p->ok = good;
  if (cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess) {
    cudaGetLastError();
    p->ok = false;
  }
  return p;
}

void tc_plan_destroy(TcPlan* p) {
  if (!p) return;
  for (int i = 0; i < 3 && p->owns_ops; ++i) {
    if (p->Ahi[i]) cudaFree(p->Ahi[i]);
    if (p->Amid[i]) cudaFree(p->Amid[i]);
    if (p->Alo[i]) cudaFree(p->Alo[i]);
  }
  if (p->E) cudaFree(p->E);
  if (p->X) cudaFree(p->X);
  if (p->S) cudaFree(p->S);
  if (p->tile_ctr) cudaFree(p->tile_ctr);
  delete p;
}

bool tc_available(const TcPlan* p) { return p && p->ok; }

TcPlan* tc_plan_create_sharing(const TcPlan* ops, int nvec, int* status) {
  if (!ops || !ops->ok) return nullptr;
  TcPlan* p = new TcPlan();
  p->N = ops->N;
  p->nvec_max = nvec;
  p->Mp = ops->Mp;
  p->Kp = ops->Kp;
  p->status = status;
  p->ok = false;
  p->owns_ops = false;
  for (int i = 0; i < 3; ++i) {
    p->Ahi[i] = ops->Ahi[i];
    p->Amid[i] = ops->Amid[i];
    p->Alo[i] = ops->Alo[i];
    p->mA_hi[i] = ops->mA_hi[i];
    p->mA_mid[i] = ops->mA_mid[i];
    p->mA_lo[i] = ops->mA_lo[i];
  }
  size_t esz = (size_t)6 * nvec * p->Kp, xsz = (size_t)3 * nvec * p->Kp;
  bool good = cudaMalloc(&p->E, 3 * esz * 2) == cudaSuccess;
  good &= cudaMalloc(&p->X, 3 * xsz * 2) == cudaSuccess;
  good &= cudaMalloc(&p->S, (size_t)6 * nvec * p->N * sizeof(float2)) == cudaSuccess;
  good &= cudaMalloc(&p->tile_ctr, 2 * sizeof(int)) == cudaSuccess && cudaMemset(p->tile_ctr, 0, 2 * sizeof(int)) == cudaSuccess;
  if (!good) {
    cudaGetLastError();
    tc_plan_destroy(p);
    return nullptr;
  }
  good = true;
  for (int t = 0; t < 3; ++t) {
    good &= make_map(&p->mE[t], p->E + t * esz, (long long)6 * nvec, p->Kp, TC_BN);
    good &= make_map(&p->mX[t], p->X + t * xsz, (long long)3 * nvec, p->Kp, TC_BN);
  }
  p->ok = good;
  return p;
}

int tc_prepare_operators(TcPlan* p, const double2* W, const double2* T, double w_scale, double t_scale, cudaStream_t s) {
  if (!p) return PC_OK;
  const long long NN = (long long)p->N * p->N, n = (long long)p->Mp * p->Kp;
  const double2* src[3] = {W, W + NN, T};
  const double sc[3] = {w_scale, w_scale, t_scale};
  for (int i = 0; i < 3; ++i) {
    k_tc_embed<<<cdiv(n, 256), 256, 0, s>>>(src[i], p->N, sc[i], p->Mp, p->Kp, p->Ahi[i], p->Amid[i], p->Alo[i]);
    PC_LAUNCH_CHECK();
  }
  return PC_OK;
}

// One persistent launch over the tiles of up to three GEMM segments.
struct TcSegSpec {
  int which, bset, col_base, ncols;
  float* C;
};
static int launch_tc_gemm(TcPlan* p, const TcSegSpec* sp, int nseg, cudaStream_t s) {
  static const int sms = [] {  // queried once; thread-safe static initialisation
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cudaGetLastError();
    return v;
  }();
  if (nseg < 1 || nseg > 3) return PC_EINVAL;
  TcGemmParams P;
  for (int w = 0; w < 3; ++w) {
    P.A[w][0] = p->mA_hi[w];
    P.A[w][1] = p->mA_mid[w];
    P.A[w][2] = p->mA_lo[w];
  }
  for (int t = 0; t < 3; ++t) {
    P.B[0][t] = p->mE[t];
    P.B[1][t] = p->mX[t];
  }
  const int mtiles = p->Mp / TC_BM;
  int tiles = 0;
  for (int g = 0; g < nseg; ++g) {
    const int nt = (sp[g].ncols + TC_BN - 1) / TC_BN;
    P.seg[g] = TcSeg{sp[g].which, sp[g].bset, sp[g].col_base, sp[g].ncols, tiles, nt, sp[g].C};
    tiles += mtiles * nt;
  }
  for (int g = nseg; g < 3; ++g) P.seg[g] = TcSeg{0, 0, 0, 0, tiles, 0, nullptr};
  P.nseg = nseg;
  P.num_kb = p->Kp / TC_BK;
  P.m_valid = 2 * p->N;
  P.mtiles = mtiles;
  P.tiles = tiles;
  P.ldc = 2LL * p->N;
  P.tile_ctr = p->tile_ctr;
  P.status = p->status;
  if (tiles == 0) return PC_OK;
  k_tc_gemm<<<std::min(tiles, sms), 192, SMEM_BYTES, s>>>(P);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int tc_apply(TcPlan* p, const float2* X, float2* AX, float2* OX, int nvec, int m, Geom g, const double* Q,
             cudaStream_t s, const float4* Kf) {
  if (!tc_available(p) || nvec > p->nvec_max) return PC_EINVAL;
  const long long n = (long long)nvec * (p->Kp / 2);
  const long long es = (long long)6 * p->nvec_max * p->Kp, xs = (long long)3 * p->nvec_max * p->Kp;
  k_tc_split_strain<<<cdiv(n, 256), 256, 0, s>>>(X, nvec, m, g, Q, Kf, p->Kp, p->E, es, p->X, xs);
  PC_LAUNCH_CHECK();
  // E column s * nvec + v holds stack s of vector v (the maps span the plan's capacity).  One
  // launch: W1 on the dilatation stack, W2 on the five deviatoric stacks (both into S), T_rho on
  // the displacements (into OX).
  const TcSegSpec seg[3] = {{0, 0, 0, nvec, (float*)p->S}, {1, 0, nvec, 5 * nvec, (float*)p->S},
                            {2, 1, 0, 3 * nvec, (float*)OX}};
  int rc = launch_tc_gemm(p, seg, 3, s);
  if (rc) return rc;
  return launch_epilogue<float>(p->S, nvec, m, g, Q, 1.0f, 1.0f, AX, s, Kf);
}
