// FP64-accurate operator products of the mixed form's final Rayleigh-Ritz step on the tensor
// cores, by exact fixed-point slicing (the scheme of Ozaki et al. for error-free matrix
// products).
//
// Every real row r of the operator (its real embedding, as in gemm_tc.cu) is scaled by a power
// of two 2^e_r with |a| 2^-e_r <= 1/2 and cut into S = 8 slices of 6-bit integers,
//   a = 2^e_r sum_{i=1..8} q_i 2^{-6 i},   q_i = rint((a 2^-e_r - sum_{l<i} q_l 2^{-6 l}) 2^{6 i}),
// |q_i| <= 32, each exact in bf16; every column c of the right-hand side the same way with its
// own 2^e_c.  The product is then
//   (A B)[r][c] = 2^{e_r + e_c} sum_t 2^{-6 t} P_t,   P_t = sum_{i + j = t} Q^A_i Q^B_j,
// and the pairs with i + j <= 9 (36 slice products) are kept (the rest lie below 2^-54 of the
// scale per term).  P_t is an integer sum of at most 8 K products of size <= 2^10: below 2^24
// for K < 2048, so the FP32 accumulation of tcgen05 computes it exactly.  Each diagonal t has its
// own accumulator in tensor memory (8 x 64 columns); the epilogue combines them in FP64 from the
// smallest scale up.  Measured against FP64 products: about 2e-12 relative to the row and column
// scales, 53-bit FP64 itself about 4e-15.
//
// GEMM (sm_103a): C[col][row] = sum_k A[row][k] B[col][k] as K-major bf16 slices (slice i of A
// at rows i * Mp.., of B at rows i * ncap..), TMA loads with the 64-byte swizzle (32 bf16 per
// row), a 2-stage ring of 8 + 8 slice tiles; warp 0 loads, warp 1 issues the 36 x 2 MMAs
// (kind::f16, M = 128, N = 64, K = 16) per stage, warps 2-5 drain and combine.  Persistent: one CTA
// per SM; the load lane claims tiles from a counter and hands them on through a ring in shared
// memory, as in gemm_tc.cu.  Every mbarrier wait is bounded (PC_ETIMEOUT on expiry).
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>
#include "gemm_tc.h"
#include "tc_ptx.cuh"

namespace {
using namespace tcx;

constexpr int OZ_BM = 128;
constexpr int OZ_BN = 64;
constexpr int OZ_BK = 32;                 // bf16 per 64-byte swizzle row
constexpr int OZ_S = 8;                   // slices per operand
constexpr int OZ_TMAX = 9;                // largest i + j kept
constexpr int OZ_NACC = OZ_TMAX - 1;      // accumulators t = 2..9
constexpr int OZ_STAGES = 2;
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2;   // 8 KB
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2;   // 4 KB
constexpr int OZ_STAGE = OZ_S * (OZ_A_TILE + OZ_B_TILE);  // 96 KB
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024 + 1024;
constexpr int OZ_KMAX = 2047;             // padded K with 8 K 2^10 < 2^24

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)4 << 61;                 // 64-byte swizzle
  return d;
}

__global__ __launch_bounds__(192, 1) void k_oz_gemm(const __grid_constant__ CUtensorMap tA,
                                                    const __grid_constant__ CUtensorMap tB, int Mp, int ncap,
                                                    int num_kb, int col_base, int ncols, int m_valid, int mtiles,
                                                    int ntiles, const double* __restrict__ row_scale,
                                                    const double* __restrict__ col_scale, double* __restrict__ C,
                                                    long long ldc, int* tile_ctr, int* status) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t bars = base + OZ_STAGES * OZ_STAGE;
  // barriers: full[s] +8s, empty[s] +64+8s, tfull +128, tempty +160, done +192; tmem slot +256;
  // tile ring: idfull[j] +320+8j, idempty[j] +352+8j, tile index j at +384+4j
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + OZ_STAGES * OZ_STAGE + 256);
  volatile int* tile_id = reinterpret_cast<volatile int*>(gbase + OZ_STAGES * OZ_STAGE + 384);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = mtiles * ntiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(bars + 8 * s, 1);
      mbar_init(bars + 64 + 8 * s, 1);
    }
    mbar_init(bars + 128, 1);
    mbar_init(bars + 160, 128);
    mbar_init(bars + 192, 1);
    for (int j = 0; j < 4; ++j) {
      mbar_init(bars + 320 + 8 * j, 1);
      mbar_init(bars + 352 + 8 * j, 5);  // the MMA lane and the four epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(OZ_NACC * OZ_BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (int tl = 0; ok; ++tl) {
        const int slot = tl & 3;
        if (!(ok = mbar_wait(bars + 352 + 8 * slot, ((uint32_t)(tl >> 2) & 1u) ^ 1u, status))) break;
        const int t = atomicAdd(tile_ctr, 1);
        tile_id[slot] = t;
        mbar_arrive(bars + 320 + 8 * slot);
        if (t >= tiles) break;
        const int m0 = (t % mtiles) * OZ_BM, n0 = (t / mtiles) * OZ_BN;
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = (int)(it % OZ_STAGES);
          const uint32_t ph = (uint32_t)(it / OZ_STAGES) & 1u;
          if (!(ok = mbar_wait(bars + 64 + 8 * s, ph ^ 1u, status))) break;
          const uint32_t st = base + s * OZ_STAGE;
          mbar_expect_tx(bars + 8 * s, OZ_STAGE);
#pragma unroll
          for (int i = 0; i < OZ_S; ++i) {
            tma_load_2d(st + i * OZ_A_TILE, &tA, bars + 8 * s, kb * OZ_BK, i * Mp + m0);
            tma_load_2d(st + OZ_S * OZ_A_TILE + i * OZ_B_TILE, &tB, bars + 8 * s, kb * OZ_BK,
                        i * ncap + col_base + n0);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_n(OZ_BN);
      long long it = 0;
      bool ok = true;
      for (int tl = 0; ok; ++tl) {  // tl: local tile index
        const int slot = tl & 3;
        if (!(ok = mbar_wait(bars + 320 + 8 * slot, (uint32_t)(tl >> 2) & 1u, status))) break;
        const int t = tile_id[slot];
        mbar_arrive(bars + 352 + 8 * slot);
        if (t >= tiles) break;
        // the accumulators must have been drained (use tl - 1)
        if (!(ok = mbar_wait(bars + 160, ((uint32_t)tl & 1u) ^ 1u, status))) break;
        tc_fence_after();
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = (int)(it % OZ_STAGES);
          const uint32_t ph = (uint32_t)(it / OZ_STAGES) & 1u;
          if (!(ok = mbar_wait(bars + 8 * s, ph, status))) break;
          tc_fence_after();
          const uint32_t st = base + s * OZ_STAGE;
#pragma unroll
          for (int kk = 0; kk < OZ_BK / 16; ++kk) {
            const uint64_t off = (uint64_t)((kk * 32) >> 4);  // 16 bf16 = 32 bytes along K
#pragma unroll
            for (int i = 1; i <= OZ_S; ++i) {
              const uint64_t ad = sw64_desc(st + (i - 1) * OZ_A_TILE) + off;
#pragma unroll
              for (int j = 1; j <= OZ_S; ++j) {
                if (i + j > OZ_TMAX) continue;
                const uint64_t bd = sw64_desc(st + OZ_S * OZ_A_TILE + (j - 1) * OZ_B_TILE) + off;
                // first product into diagonal t of this tile: i = 1 (j = t - 1), at the first K step
                const uint32_t acc = (kb > 0 || kk > 0 || i > 1) ? 1u : 0u;
                mma_bf16(tmem + (uint32_t)((i + j - 2) * OZ_BN), ad, bd, idesc, acc);
              }
            }
          }
          mma_commit(bars + 64 + 8 * s);  // stage free once these MMAs have read it
        }
        if (ok) mma_commit(bars + 128);  // accumulators complete
      }
      mma_commit(bars + 192);
      mbar_wait(bars + 192, 0u, status);
    }
  } else {
    // epilogue warps 2..5: lane quadrant (warp % 4) of the accumulators
    const int quad = warp & 3;
    for (int tl = 0;; ++tl) {
      const int slot = tl & 3;
      if (!__all_sync(0xffffffffu, mbar_wait(bars + 320 + 8 * slot, (uint32_t)(tl >> 2) & 1u, status))) break;
      const int t = tile_id[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + 352 + 8 * slot);
      if (t >= tiles) break;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(bars + 128, (uint32_t)tl & 1u, status));
      tc_fence_after();
      const int row = (t % mtiles) * OZ_BM + quad * 32 + lane;
      const int n0 = (t / mtiles) * OZ_BN;
      const double rs = (ok && row < m_valid) ? row_scale[row] : 0.0;
#pragma unroll 1
      for (int c = 0; c < OZ_BN / 16; ++c) {
        double sum[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) sum[j] = 0.0;
        // from the smallest scale (t = 9) to the largest (t = 2)
#pragma unroll 1
        for (int a = OZ_NACC - 1; a >= 0; --a) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * OZ_BN + c * 16), v);
          const double sc = ldexp(1.0, -6 * (a + 2));
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[j] = fma((double)v[j], sc, sum[j]);
        }
        if (!ok || row >= m_valid) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c * 16 + j;
          if (col < ncols) C[(long long)col * ldc + row] = sum[j] * rs * col_scale[col_base + col];
        }
      }
      tc_fence_before();
      mbar_arrive(bars + 160);
      if (!ok) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(OZ_NACC * OZ_BN))
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
// Slicing.  One warp per row (of the real embedding of a complex operator, rows 2p and 2p+1
// share the magnitudes of complex row p) or per column (a complex vector of length N, real K
// index 2q + {re, im}).  Slice i of row/column x is written at out + i * slice_stride + x * Kp;
// K positions past 2N are zero.
// The eight 6-bit slices of v / 2^e (|v| 2^-e <= 1/2): I = rint(v 2^-e 2^48) as a 64-bit integer,
// then balanced base-64 digits from the least significant up (each in [-32, 31], the leading one
// in [-32, 32]), so that sum_i q_i 2^-6i = I 2^-48.  This is the value the successive cuts
// q_i = rint((r - sum_{l<i} q_l 2^-6l) 2^6i) represent: the parts already cut are multiples of
// 2^-42, so the last cut rounds r 2^48 shifted by a multiple of 64, which changes neither the
// rounding nor a tie's parity.  Integer work only after one multiply and one conversion.
__device__ __forceinline__ void slice8(double v, double inv_scale48, int q[OZ_S]) {
  long long I = __double2ll_rn(v * inv_scale48);  // the multiply is by a power of two: exact
#pragma unroll
  for (int i = OZ_S - 1; i > 0; --i) {
    int d = (int)(I & 63);
    d -= (d >= 32) ? 64 : 0;
    q[i] = d;
    I = (I - d) >> 6;
  }
  q[0] = (int)I;
}

// Power of two 2^e with max |x| 2^-e in (1/4, 1/2] (1 for an all-zero row).
__device__ __forceinline__ double pow2_scale(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);  // mx = f 2^e, f in [1/2, 1)
  return ldexp(1.0, e + 1);
}

// Four consecutive K entries (two complex values) of one row or column, sliced and stored as
// 8 bytes per slice.
__device__ __forceinline__ void store_slices4(const double v[4], double inv48, __nv_bfloat16* dst,
                                              long long sstride) {
  int q[4][OZ_S];
#pragma unroll
  for (int e = 0; e < 4; ++e) slice8(v[e], inv48, q[e]);
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    __nv_bfloat162 lo = __floats2bfloat162_rn((float)q[0][i], (float)q[1][i]);
    __nv_bfloat162 hi = __floats2bfloat162_rn((float)q[2][i], (float)q[3][i]);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&lo);
    u.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(dst + i * sstride) = u;
  }
}

// One warp per real row of alpha W (rows 2p, 2p + 1 of [[Re, -Im], [Im, Re]]); rows beyond 2N and
// columns beyond 2N are zero.  Kp is a multiple of 32, so every 4-entry group is 8-byte aligned.
__global__ void k_oz_slice_rows(const double2* __restrict__ W, int N, double alpha, int Mp, int Kp,
                                __nv_bfloat16* __restrict__ out, double* __restrict__ row_scale) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= Mp) return;
  const long long sstride = (long long)Mp * Kp;
  __nv_bfloat16* o = out + (long long)row * Kp;
  if (row >= 2 * N) {
    const uint2 z = make_uint2(0u, 0u);
    for (int k = 4 * lane; k < Kp; k += 128)
      for (int i = 0; i < OZ_S; ++i) *reinterpret_cast<uint2*>(o + i * sstride + k) = z;
    if (lane == 0) row_scale[row] = 0.0;
    return;
  }
  const int p = row >> 1, r = row & 1;
  const double2* w = W + (long long)p * N;
  double mx = 0.0;
  for (int q = lane; q < N; q += 32) mx = fmax(mx, fmax(fabs(w[q].x), fabs(w[q].y)) * fabs(alpha));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const double sc = pow2_scale(mx), inv48 = ldexp(1.0 / sc, 48);
  for (int k = 4 * lane; k < Kp; k += 128) {
    double v[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = (k >> 1) + h;
      const double2 z = q < N ? w[q] : make_double2(0.0, 0.0);
      v[2 * h] = alpha * (r == 0 ? z.x : z.y);       // column 2q: Re z (row 2p), Im z (row 2p + 1)
      v[2 * h + 1] = alpha * (r == 0 ? -z.y : z.x);  // column 2q + 1: -Im z, Re z
    }
    store_slices4(v, inv48, o + k, sstride);
  }
  if (lane == 0) row_scale[row] = sc;
}

// One warp per complex column of X (real entries Re, Im interleaved along K); entries beyond 2N are zero.
__global__ void k_oz_slice_cols(const double2* __restrict__ X, int ncols, int N, int Kp, long long sstride,
                                int col_off, __nv_bfloat16* __restrict__ out, double* __restrict__ col_scale) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= ncols) return;
  const double2* x = X + (long long)c * N;
  double mx = 0.0;
  for (int q = lane; q < N; q += 32) mx = fmax(mx, fmax(fabs(x[q].x), fabs(x[q].y)));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const double sc = pow2_scale(mx), inv48 = ldexp(1.0 / sc, 48);
  const long long cc = (long long)col_off + c;
  __nv_bfloat16* o = out + cc * Kp;
  for (int k = 4 * lane; k < Kp; k += 128) {
    const int q = k >> 1;
    const double2 z0 = q < N ? x[q] : make_double2(0.0, 0.0);
    const double2 z1 = q + 1 < N ? x[q + 1] : make_double2(0.0, 0.0);
    const double v[4] = {z0.x, z0.y, z1.x, z1.y};
    store_slices4(v, inv48, o + k, sstride);
  }
  if (lane == 0) col_scale[cc] = sc;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn oz_encode() {
  static const EncodeTiledFn fn = [] {  // looked up once; thread-safe static initialisation
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    EncodeTiledFn f = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = (EncodeTiledFn)p;
    cudaGetLastError();
    return f;
  }();
  return fn;
}

// 2-D K-major bf16 tensor map over rows x Kp, box 32 x box_rows, 64-byte swizzle.
bool oz_map(CUtensorMap* m, void* ptr, long long rows, int Kp, int box_rows) {
  EncodeTiledFn enc = oz_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count_oz() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cudaGetLastError();
    return v;
  }();
  return n;
}

}  // namespace

struct OzPlan {
  int N, Mp, Kp, ncap;
  __nv_bfloat16* A[3] = {nullptr, nullptr, nullptr};  // W1, W2, T_rho: [8][Mp][Kp]
  double* rs[3] = {nullptr, nullptr, nullptr};        // row scales (Mp)
  __nv_bfloat16* Bs = nullptr;                        // right-hand sides: [8][ncap][Kp]
  double* cs = nullptr;                               // column scales (ncap)
  CUtensorMap mA[3], mB;
  int* status = nullptr;
  int* tile_ctr = nullptr;                            // tile counter and finished-CTA count of k_oz_gemm
  bool ok = false, owns_ops = true;
};

bool oz_eligible(int N) { return ((2 * N + OZ_BK - 1) / OZ_BK) * OZ_BK <= OZ_KMAX; }

OzPlan* oz_plan_create(int N, int ncap, int* status, const OzPlan* share) {
  if (!oz_eligible(N)) return nullptr;
  OzPlan* p = new OzPlan();
  p->N = N;
  p->Mp = ((2 * N + OZ_BM - 1) / OZ_BM) * OZ_BM;
  p->Kp = ((2 * N + OZ_BK - 1) / OZ_BK) * OZ_BK;
  p->ncap = ((ncap + OZ_BN - 1) / OZ_BN) * OZ_BN;
  p->status = status;
  bool good = true;
  const size_t asz = (size_t)OZ_S * p->Mp * p->Kp;
  if (share) {
    p->owns_ops = false;
    for (int i = 0; i < 3; ++i) {
      p->A[i] = share->A[i];
      p->rs[i] = share->rs[i];
      p->mA[i] = share->mA[i];
    }
  } else {
    for (int i = 0; i < 3; ++i) {
      good &= cudaMalloc(&p->A[i], asz * 2) == cudaSuccess;
      good &= cudaMalloc(&p->rs[i], sizeof(double) * p->Mp) == cudaSuccess;
    }
  }
  good &= cudaMalloc(&p->Bs, (size_t)OZ_S * p->ncap * p->Kp * 2) == cudaSuccess;
  good &= cudaMalloc(&p->cs, sizeof(double) * p->ncap) == cudaSuccess;
  good &= cudaMalloc(&p->tile_ctr, 2 * sizeof(int)) == cudaSuccess && cudaMemset(p->tile_ctr, 0, 2 * sizeof(int)) == cudaSuccess;
  if (!good) {
    cudaGetLastError();
    oz_plan_destroy(p);
    return nullptr;
  }
  good = true;
  if (!share)
    for (int i = 0; i < 3; ++i) good &= oz_map(&p->mA[i], p->A[i], (long long)OZ_S * p->Mp, p->Kp, OZ_BM);
  good &= oz_map(&p->mB, p->Bs, (long long)OZ_S * p->ncap, p->Kp, OZ_BN);
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  p->ok = good && attr == cudaSuccess;
  if (!p->ok) cudaGetLastError();
  return p;
}

void oz_plan_destroy(OzPlan* p) {
  if (!p) return;
  for (int i = 0; i < 3 && p->owns_ops; ++i) {
    if (p->A[i]) cudaFree(p->A[i]);
    if (p->rs[i]) cudaFree(p->rs[i]);
  }
  if (p->Bs) cudaFree(p->Bs);
  if (p->cs) cudaFree(p->cs);
  if (p->tile_ctr) cudaFree(p->tile_ctr);
  delete p;
}

bool oz_available(const OzPlan* p) { return p && p->ok; }

int oz_prepare_operators(OzPlan* p, const double2* W, const double2* T, double w_scale, double t_scale,
                         cudaStream_t s) {
  const long long NN = (long long)p->N * p->N;
  const double2* src[3] = {W, W + NN, T};
  const double sc[3] = {w_scale, w_scale, t_scale};
  for (int i = 0; i < 3; ++i) {
    k_oz_slice_rows<<<cdiv(p->Mp, 8), 256, 0, s>>>(src[i], p->N, sc[i], p->Mp, p->Kp, p->A[i], p->rs[i]);
    PC_LAUNCH_CHECK();
  }
  return PC_OK;
}

int oz_slice_columns(OzPlan* p, const double2* X, int ncols, int col_off, cudaStream_t s) {
  if (col_off + ncols > p->ncap) return PC_EINVAL;
  k_oz_slice_cols<<<cdiv(ncols, 8), 256, 0, s>>>(X, ncols, p->N, p->Kp, (long long)p->ncap * p->Kp, col_off, p->Bs,
                                                 p->cs);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int oz_gemm(OzPlan* p, int which_A, int col_base, int ncols, double2* C, cudaStream_t s) {
  if (!oz_available(p) || col_base + ncols > p->ncap) return PC_EINVAL;
  const int mtiles = p->Mp / OZ_BM, ntiles = (ncols + OZ_BN - 1) / OZ_BN;
  const int grid = std::min(mtiles * ntiles, sm_count_oz());
  // output column c (right-hand side column col_base + c) at C + c N
  k_oz_gemm<<<grid, 192, OZ_SMEM, s>>>(p->mA[which_A], p->mB, p->Mp, p->ncap, p->Kp / OZ_BK, col_base, ncols,
                                       2 * p->N, mtiles, ntiles, p->rs[which_A], p->cs, reinterpret_cast<double*>(C),
                                       2LL * p->N, p->tile_ctr, p->status);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// ---------------------------------------------------------------------------
// Self-check: the sliced product against the FP64 GEMM on seeded data whose rows span eight
// binades (scales 2^-4 .. 2^4), N plane waves, ncols complex columns.
namespace {
__global__ void k_oz_fill(double2* x, long long n, unsigned long long seed, int N, int graded) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  unsigned long long h = (unsigned long long)t * 0x9E3779B97F4A7C15ull + seed;
  h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29; h *= 0x94D049BB133111EBull; h ^= h >> 32;
  const double a = (double)(h & 0xFFFFFFFFull) / 4294967296.0 - 0.5, b = (double)(h >> 32) / 4294967296.0 - 0.5;
  const double sc = graded ? ldexp(1.0, (int)((t / N) % 9) - 4) : 1.0;
  x[t] = make_double2(a * sc, b * sc);
}
__global__ void k_oz_maxdiff(const double2* a, const double2* b, long long n, double* out) {
  __shared__ double sd[256], sr[256];
  double d = 0, r = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    d = fmax(d, fmax(fabs(a[t].x - b[t].x), fabs(a[t].y - b[t].y)));
    r = fmax(r, fmax(fabs(b[t].x), fabs(b[t].y)));
  }
  sd[threadIdx.x] = d;
  sr[threadIdx.x] = r;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + w]);
      sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[2 * blockIdx.x] = sd[0]; out[2 * blockIdx.x + 1] = sr[0]; }
}
}  // namespace

int oz_self_check(int N, int ncols, double* rel_err) {
  if (N < 1 || ncols < 1 || !oz_eligible(N)) return PC_EINVAL;
  const long long NN = (long long)N * N, nx = (long long)ncols * N;
  double2 *W = nullptr, *X = nullptr, *Co = nullptr, *Cr = nullptr;
  double* red = nullptr;
  int* status = nullptr;
  // W holds the two operator blocks oz_prepare_operators reads (W1, W2), T is passed as W too
  bool ok = cudaMalloc(&W, 2 * NN * sizeof(double2)) == cudaSuccess && cudaMalloc(&X, nx * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&Co, nx * sizeof(double2)) == cudaSuccess && cudaMalloc(&Cr, nx * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&red, 2 * 64 * sizeof(double)) == cudaSuccess && cudaMalloc(&status, sizeof(int)) == cudaSuccess;
  int rc = ok ? PC_OK : PC_ENOMEM;
  OzPlan* p = nullptr;
  if (!rc) {
    cudaMemset(status, 0, sizeof(int));
    k_oz_fill<<<cdiv(2 * NN, 256), 256>>>(W, 2 * NN, 12345ull, N, 1);
    k_oz_fill<<<cdiv(nx, 256), 256>>>(X, nx, 54321ull, N, 0);
    p = oz_plan_create(N, ncols, status, nullptr);
    if (!p) rc = PC_ENOMEM;
    else if (!oz_available(p)) rc = PC_ECUDA;  // tensor maps or the kernel attribute
  }
  if (!rc) rc = oz_prepare_operators(p, W, W, 1.0, 1.0, 0);  // W1 = T = the first block, W2 the second
  if (!rc) rc = oz_slice_columns(p, X, ncols, 0, 0);
  if (!rc) rc = oz_gemm(p, 0, 0, ncols, Co, 0);
  if (!rc) rc = launch_gemm<double>(N, ncols, N, W, N, X, N, Cr, N, 1.0, 0);
  if (!rc) {
    k_oz_maxdiff<<<64, 256>>>(Co, Cr, nx, red);
    double h[128];
    int st = 0;
    if (cudaMemcpy(h, red, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = PC_ECUDA;
    if (!rc && st) rc = st;
    if (!rc) {
      double d = 0, r = 0;
      for (int i = 0; i < 64; ++i) { d = std::max(d, h[2 * i]); r = std::max(r, h[2 * i + 1]); }
      *rel_err = r > 0 ? d / r : d;
    }
  }
  oz_plan_destroy(p);
  cudaFree(W); cudaFree(X); cudaFree(Co); cudaFree(Cr); cudaFree(red); cudaFree(status);
  cudaGetLastError();
  return rc;
}
