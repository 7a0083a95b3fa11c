// Tall-skinny products of the block iteration on the tensor cores (sm_103a), FP32 data:
//   gram   -- G_part[k][split] = A^H B over one range of the 3N rows (A: ca columns, B: cb columns)
//   update -- out_h = sum_b in_b C_h[b] (+ in_last when the last block is the identity), for one
//             or two coefficient sets h sharing the inputs
// Both are dense complex contractions.  A complex column stored as interleaved (re, im) pairs is
// a real vector; with b~ = (Im b, -Re b) per entry, Re(a^H b) = a . b and Im(a^H b) = a . b~, so
// the Gram matrix is the real product A^T [B | B~].  For the update, row r of the inputs is the
// real vector (Re s_i, Im s_i)_i and each output column is two real columns of coefficients,
// (Re c, -Im c) for the real part and (Im c, Re c) for the imaginary part.
//
// The FP32 operands are split exactly into three bf16 slices in shared memory by the staging
// warps (x = hi + mid + lo, 8 significand bits each); the six slice products of order at most 2^-16
// (hh, hm, mh, hl, mm, lh) are accumulated in FP32 in tensor memory by tcgen05.mma
// (kind::f16, M = 128, K = 16).  Staging is double-buffered against the MMAs with mbarriers;
// every wait is bounded and records PC_ETIMEOUT in the status word when it expires.
#include <math.h>
#include <string.h>
#include <vector>
#include "gemm_tc.h"
#include "kernels.h"
#include "tc_ptx.cuh"

using namespace tcx;

std::atomic<int> g_tc_tall{1};  // tensor-core Gram and update kernels for FP32 data (0: CUDA cores,
                                // switched only by pc_check_tensor_kernels for its reference run)

namespace {

constexpr int A_SLICE = 128 * 128;  // 128 rows x 64 bf16 (one 128-byte swizzle atom along K)

int sm_count() {
  static const int n = [] {  // queried once; thread-safe static initialisation
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cudaGetLastError();
    return v;
  }();
  return n;
}

// Splits of a work range into parts so that ceil(units * parts / sms) waves of
// ceil(len / parts) steps are as short as possible (one CTA per SM).
int best_split(int units, int len, int max_parts) {
  const int sms = sm_count();
  int best = 1;
  long long best_t = -1;
  for (int p = 1; p <= max_parts && p <= len; ++p) {
    long long waves = (units * (long long)p + sms - 1) / sms;
    long long t = waves * ((len + p - 1) / p);
    if (best_t < 0 || t < best_t) { best_t = t; best = p; }
  }
  return best;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// (re, im) bf16 pair -> (im, -re): swap the halves, then flip the sign of the upper half.
__device__ __forceinline__ uint32_t rot_pair(uint32_t w) { return __funnelshift_l(w, w, 16) ^ 0x80000000u; }

// ---------------------------------------------------------------------------
// Gram products.
constexpr int G_THREADS = 544;  // warps 0-15 stage operands (warps 0-3 also drain), warp 16 issues MMAs
constexpr int G_PRODUCERS = 512;
constexpr int G_MMA_WARP = 16;
constexpr int G_BROWS = 144;    // B rows: cb real parts + cb rotated parts, cb <= 72
constexpr int G_B_SLICE = G_BROWS * 128;
constexpr int G_STAGE = 3 * (A_SLICE + G_B_SLICE);
constexpr int G_SMEM = 2 * G_STAGE + 256 + 1024;
constexpr int G_MAXI = (144 * 16 + G_PRODUCERS - 1) / G_PRODUCERS;  // staged items per thread and stage

struct TcGramArgs {
  const float2* A[3];
  const float2* B[3];
  int na, nbk, m, n3;
  int nsplit, rows_per_split;  // rows_per_split: a multiple of 32
  float2* part;
  int* status;
};

__global__ __launch_bounds__(G_THREADS, 1) void k_tc_gram(TcGramArgs a) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t bars = base + 2 * G_STAGE;  // full[s] +8s, empty[s] +16+8s, accumulator +32
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + 2 * G_STAGE + 64);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x, split = blockIdx.y;
  const int ca = a.na * a.m, cb = a.nbk * a.m;
  const int NP = ((2 * cb + 15) / 16) * 16;
  const long long kofs = (long long)k * a.m * a.n3;
  const int r_begin = split * a.rows_per_split;
  const int r_end = min(a.n3, r_begin + a.rows_per_split);
  const int nst = r_end > r_begin ? (r_end - r_begin + 31) / 32 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(bars + 8 * s, G_PRODUCERS);
      mbar_init(bars + 16 + 8 * s, 1);
    }
    mbar_init(bars + 32, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == G_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < G_MMA_WARP) {
    // Every load of a stage is issued before any is used, and the loads of stage it + 1 are
    // in flight while stage it is split and stored: one HBM latency per stage, overlapped.
    const int nitems = (ca + cb) * 16;
    // Item u of this thread is the same column and row pair in every stage: its source
    // column and its shared-memory offsets are computed once.
    const float2* colp[G_MAXI];
    uint32_t off1[G_MAXI], off2[G_MAXI];
    int qq[G_MAXI];
#pragma unroll
    for (int u = 0; u < G_MAXI; ++u) {
      const int e = threadIdx.x + u * G_PRODUCERS;
      const int c = e < nitems ? e >> 4 : 0, q = e & 15;
      const bool isA = c < ca;
      const int col = isA ? c : c - ca;
      const int b = col / a.m;
      const float2* base_p = isA ? (b == 0 ? a.A[0] : (b == 1 ? a.A[1] : a.A[2]))
                                 : (b == 0 ? a.B[0] : (b == 1 ? a.B[1] : a.B[2]));
      colp[u] = base_p + kofs + (long long)(col - b * a.m) * a.n3;
      qq[u] = e < nitems ? 2 * q : 1 << 30;  // rows of an unused item never pass the bound
      off1[u] = isA ? sw128_offset(col, 8 * q) : 3 * A_SLICE + sw128_offset(col, 8 * q);
      off2[u] = isA ? 0xffffffffu : 3 * A_SLICE + sw128_offset(cb + col, 8 * q);
    }
    float2 va[2][G_MAXI], vb[2][G_MAXI];
    auto fetch = [&](int it, float2 (&x0)[G_MAXI], float2 (&x1)[G_MAXI]) {
      const int r0 = r_begin + it * 32;
#pragma unroll
      for (int u = 0; u < G_MAXI; ++u) {
        const int r = r0 + qq[u];
        x0[u] = r < r_end ? colp[u][r] : make_float2(0.f, 0.f);
        x1[u] = r + 1 < r_end ? colp[u][r + 1] : make_float2(0.f, 0.f);
        // stage it + 2 into L2 (no registers held), so its loads one stage later hit there
        if (r + 64 < r_end) prefetch_l2(colp[u] + r + 64);
      }
    };
    auto stash = [&](int it, const float2 (&x0)[G_MAXI], const float2 (&x1)[G_MAXI]) {
      unsigned char* stp = gbase + (it & 1) * G_STAGE;
#pragma unroll
      for (int u = 0; u < G_MAXI; ++u) {
        if (qq[u] < 32) {
          uint2 h, mi, lo;
          split4_exact(x0[u].x, x0[u].y, x1[u].x, x1[u].y, h, mi, lo);
          const uint32_t o1 = off1[u], o2 = off2[u];
          if (o2 == 0xffffffffu) {
            *reinterpret_cast<uint2*>(stp + o1) = h;
            *reinterpret_cast<uint2*>(stp + A_SLICE + o1) = mi;
            *reinterpret_cast<uint2*>(stp + 2 * A_SLICE + o1) = lo;
          } else {
            *reinterpret_cast<uint2*>(stp + o1) = h;
            *reinterpret_cast<uint2*>(stp + G_B_SLICE + o1) = mi;
            *reinterpret_cast<uint2*>(stp + 2 * G_B_SLICE + o1) = lo;
            *reinterpret_cast<uint2*>(stp + o2) = make_uint2(rot_pair(h.x), rot_pair(h.y));
            *reinterpret_cast<uint2*>(stp + G_B_SLICE + o2) = make_uint2(rot_pair(mi.x), rot_pair(mi.y));
            *reinterpret_cast<uint2*>(stp + 2 * G_B_SLICE + o2) = make_uint2(rot_pair(lo.x), rot_pair(lo.y));
          }
        }
      }
    };
    if (nst > 0) fetch(0, va[0], vb[0]);
    for (int it = 0; it < nst; it += 2) {
      // even stage from buffer 0, odd stage from buffer 1 (register arrays stay statically indexed)
      if (it + 1 < nst) fetch(it + 1, va[1], vb[1]);
      if (!mbar_wait(bars + 16, ((uint32_t)(it >> 1) & 1u) ^ 1u, a.status)) break;
      stash(it, va[0], vb[0]);
      fence_async_smem();
      mbar_arrive(bars);
      if (it + 1 >= nst) break;
      if (it + 2 < nst) fetch(it + 2, va[0], vb[0]);
      if (!mbar_wait(bars + 24, ((uint32_t)((it + 1) >> 1) & 1u) ^ 1u, a.status)) break;
      stash(it + 1, va[1], vb[1]);
      fence_async_smem();
      mbar_arrive(bars + 8);
    }
  } else if (lane == 0) {
    const uint32_t idesc = idesc_bf16_n(NP);
    for (int it = 0; it < nst; ++it) {
      const int s = it & 1;
      const uint32_t ph = (uint32_t)(it >> 1) & 1u;
      if (!mbar_wait(bars + 8 * s, ph, a.status)) break;
      tc_fence_after();
      const uint32_t st = base + s * G_STAGE;
      const uint64_t ah = sw128_desc(st), am = sw128_desc(st + A_SLICE), al = sw128_desc(st + 2 * A_SLICE);
      const uint32_t sb = st + 3 * A_SLICE;
      const uint64_t bh = sw128_desc(sb), bm = sw128_desc(sb + G_B_SLICE), bl = sw128_desc(sb + 2 * G_B_SLICE);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t off = (uint64_t)(2 * kk);  // 16 bf16 = 32 bytes along K
        mma_bf16(tmem, ah + off, bh + off, idesc, (it > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, ah + off, bm + off, idesc, 1u);
        mma_bf16(tmem, am + off, bh + off, idesc, 1u);
        mma_bf16(tmem, ah + off, bl + off, idesc, 1u);
        mma_bf16(tmem, am + off, bm + off, idesc, 1u);
        mma_bf16(tmem, al + off, bh + off, idesc, 1u);
      }
      mma_commit(bars + 16 + 8 * s);
    }
    mma_commit(bars + 32);
  }
  // drain: warps 0-3 copy their accumulator lanes to shared memory (stage 0 is free once
  // every MMA has completed), then the whole CTA writes the partial Gram matrix
  const int ld = NP + 1;
  float* stage = reinterpret_cast<float*>(gbase);
  if (warp < 4) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bars + 32, 0u, a.status));
    tc_fence_after();
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) stage[row * ld + c0 + j] = (ok && nst > 0) ? v[j] : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  float2* out = a.part + ((long long)k * a.nsplit + split) * ca * cb;
  for (int e = threadIdx.x; e < ca * cb; e += G_THREADS) {
    const int i = e / cb, j = e % cb;
    out[e] = make_float2(stage[i * ld + j], stage[i * ld + cb + j]);
  }
  if (warp == G_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Basis updates.
constexpr int U_THREADS = 672;  // warps 0-15 stage, warps 16-19 drain, warp 20 issues MMAs
constexpr int U_PRODUCERS = 512;
constexpr int U_EPI_WARP = 16, U_MMA_WARP = 20;
constexpr int U_EPI = 128;
constexpr int U_KMAX = 192;     // padded real K (2 * 72 input columns -> 144 -> 3 atoms)
constexpr int U_NMAX = 96;
constexpr int U_BOP = 3 * U_NMAX * U_KMAX * 2;  // coefficient operand, three slices
constexpr int U_STAGE = 3 * A_SLICE;
constexpr int U_SMEM = U_BOP + 2 * U_STAGE + 256 + 72 * 8 + 1024;  // + input column table
constexpr int U_MAXI = 128 * 16 / U_PRODUCERS;  // staged items per thread and stage

struct TcUpdateArgs {
  const float2* in[3][3];
  float2* out[2][3];           // [coefficient set][triplet]
  const float2* C[2];
  long long cstride;
  int cld, nblk, identity_last, m, mout, n3;
  long long in_kstride, out_kstride;
  int tiles, tiles_per_cta;
  int* status;
};

template <int MOUT, int NC>
__global__ __launch_bounds__(U_THREADS, 1) void k_tc_update(TcUpdateArgs a) {
  constexpr int NP = ((2 * MOUT * NC + 15) / 16) * 16;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t bop = base;
  const uint32_t stg = base + U_BOP;
  // barriers: full[s] +8s, empty[s] +16+8s, tfull[b] +32+8b, tempty[b] +48+8b, done +64
  const uint32_t bars = stg + 2 * U_STAGE;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + U_BOP + 2 * U_STAGE + 128);
  const float2** colp = reinterpret_cast<const float2**>(gbase + U_BOP + 2 * U_STAGE + 256);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x, t = blockIdx.y;
  const int ncols = a.nblk * a.m;           // complex input columns
  const int Kt = 2 * ncols;                 // real K
  const int nat = (Kt + 63) / 64;           // K atoms
  const int tile0 = blockIdx.z * a.tiles_per_cta;
  const int ntl = max(0, min(a.tiles, tile0 + a.tiles_per_cta) - tile0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(bars + 8 * s, U_PRODUCERS);
      mbar_init(bars + 16 + 8 * s, 1);
      mbar_init(bars + 32 + 8 * s, 1);
      mbar_init(bars + 48 + 8 * s, U_EPI);
    }
    mbar_init(bars + 64, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == U_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // coefficient operand: row jj = h * 2 MOUT + part * MOUT + j, K = 2 i + {0, 1}.  The
  // coefficients are first copied to the (not yet used) staging area with all loads in flight.
  const int crows = a.identity_last ? (a.nblk - 1) * a.m : ncols;
  float2* cs = reinterpret_cast<float2*>(gbase + U_BOP);  // [h][i][j], j < MOUT
  {
    constexpr int CMAX = (2 * 72 * 24 + U_THREADS - 1) / U_THREADS;
    float2 cv[CMAX];
    const int ncel = NC * crows * MOUT;
#pragma unroll
    for (int u = 0; u < CMAX; ++u) {
      const int e = threadIdx.x + u * U_THREADS;
      cv[u] = make_float2(0.f, 0.f);
      if (e < ncel) {
        const int h = e / (crows * MOUT), rem = e % (crows * MOUT), i = rem / MOUT, j = rem % MOUT;
        if (j < a.mout) cv[u] = (h == 0 ? a.C[0] : a.C[1])[(long long)k * a.cstride + (long long)i * a.cld + j];
      }
    }
#pragma unroll
    for (int u = 0; u < CMAX; ++u) {
      const int e = threadIdx.x + u * U_THREADS;
      if (e < ncel) cs[e] = cv[u];
    }
  }
  __syncthreads();
  {
    const int npairs = NP * (nat * 32);
    for (int e = threadIdx.x; e < npairs; e += U_THREADS) {
      const int jj = e / (nat * 32), i = e % (nat * 32);
      const int h = jj / (2 * MOUT), rem = jj % (2 * MOUT), part = rem / MOUT, j = rem % MOUT;
      float x0 = 0.f, x1 = 0.f;
      if (h < NC && j < a.mout && i < ncols) {
        float2 c;
        if (i >= crows) c = make_float2((i - crows) == j ? 1.f : 0.f, 0.f);  // identity block
        else c = cs[(h * crows + i) * MOUT + j];
        if (part == 0) { x0 = c.x; x1 = -c.y; }
        else { x0 = c.y; x1 = c.x; }
      }
      uint32_t w[3];
      split2_exact(x0, x1, w[0], w[1], w[2]);
      const int at = i >> 5;                 // atom of K = 2i
      const uint32_t off = sw128_offset(jj, 4 * (i & 31));
#pragma unroll
      for (int sl = 0; sl < 3; ++sl)
        *reinterpret_cast<uint32_t*>(gbase + (size_t)(sl * nat + at) * NP * 128 + off) = w[sl];
    }
  }
  // first element of every input column of this (k, triplet)
  for (int i = threadIdx.x; i < ncols; i += U_THREADS) {
    const int b = i / a.m;
    colp[i] = a.in[t][b] + (long long)k * a.in_kstride + (long long)(i - b * a.m) * a.n3;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nstage = ntl * nat;

  if (warp < U_EPI_WARP) {
    // All loads of a stage are issued together; the next stage's loads are in flight while
    // the current one is split and stored.  A warp covers 8 rows x 4 column pairs, so its
    // 8-byte stores under the 128-byte swizzle touch every bank exactly twice (no conflicts).
    float2 pa[2][U_MAXI], pb[2][U_MAXI];
    // item u of this thread: the same row and K column pair in every stage
    int rr_u[U_MAXI], ip_u[U_MAXI];
    uint32_t off_u[U_MAXI];
#pragma unroll
    for (int u = 0; u < U_MAXI; ++u) {
      const int e = threadIdx.x + u * U_PRODUCERS;
      rr_u[u] = 8 * ((e >> 5) & 15) + (e & 7);
      ip_u[u] = 4 * (e >> 9) + ((e >> 3) & 3);
      off_u[u] = sw128_offset(rr_u[u], 8 * ip_u[u]);
    }
    auto fetch = [&](int it, float2 (&x0)[U_MAXI], float2 (&x1)[U_MAXI]) {
      const int tl = it / nat, at = it % nat;
      const int r0 = (tile0 + tl) * 128;
      const int nip = min(64, ((Kt - 64 * at + 15) / 16) * 16) / 4;
#pragma unroll
      for (int u = 0; u < U_MAXI; ++u) {
        x0[u] = make_float2(0.f, 0.f);
        x1[u] = make_float2(0.f, 0.f);
        const int r = r0 + rr_u[u];
        const int i0 = 32 * at + 2 * ip_u[u];
        if (ip_u[u] < nip && r < a.n3) {
          if (i0 < ncols) x0[u] = colp[i0][r];
          if (i0 + 1 < ncols) x1[u] = colp[i0 + 1][r];
        }
      }
      // stage it + 2 into L2 (no registers held), so its loads one stage later hit there
      const int it2 = it + 2;
      if (it2 < nstage) {
        const int tl2 = it2 / nat, at2 = it2 % nat;
        const int r02 = (tile0 + tl2) * 128;
        const int nip2 = min(64, ((Kt - 64 * at2 + 15) / 16) * 16) / 4;
#pragma unroll
        for (int u = 0; u < U_MAXI; ++u) {
          const int r = r02 + rr_u[u];
          const int i0 = 32 * at2 + 2 * ip_u[u];
          if (ip_u[u] < nip2 && r < a.n3 && i0 < ncols) prefetch_l2(colp[i0] + r);
        }
      }
    };
    auto stash = [&](int it, const float2 (&x0)[U_MAXI], const float2 (&x1)[U_MAXI]) {
      const int at = it % nat;
      const int nip = min(64, ((Kt - 64 * at + 15) / 16) * 16) / 4;
      unsigned char* stp = gbase + U_BOP + (it & 1) * U_STAGE;
#pragma unroll
      for (int u = 0; u < U_MAXI; ++u) {
        if (ip_u[u] < nip) {
          uint2 h, mi, lo;
          split4_exact(x0[u].x, x0[u].y, x1[u].x, x1[u].y, h, mi, lo);
          *reinterpret_cast<uint2*>(stp + off_u[u]) = h;
          *reinterpret_cast<uint2*>(stp + A_SLICE + off_u[u]) = mi;
          *reinterpret_cast<uint2*>(stp + 2 * A_SLICE + off_u[u]) = lo;
        }
      }
    };
    if (nstage > 0) fetch(0, pa[0], pb[0]);
    for (int it = 0; it < nstage; it += 2) {
      if (it + 1 < nstage) fetch(it + 1, pa[1], pb[1]);
      if (!mbar_wait(bars + 16, ((uint32_t)(it >> 1) & 1u) ^ 1u, a.status)) break;
      stash(it, pa[0], pb[0]);
      fence_async_smem();
      mbar_arrive(bars);
      if (it + 1 >= nstage) break;
      if (it + 2 < nstage) fetch(it + 2, pa[0], pb[0]);
      if (!mbar_wait(bars + 24, ((uint32_t)((it + 1) >> 1) & 1u) ^ 1u, a.status)) break;
      stash(it + 1, pa[1], pb[1]);
      fence_async_smem();
      mbar_arrive(bars + 8);
    }
  } else if (warp < U_MMA_WARP) {
    const int quad = warp & 3;
    const int r_in = quad * 32 + lane;
    for (int tl = 0; tl < ntl; ++tl) {
      const int b = tl & 1;
      const uint32_t ph = (uint32_t)(tl >> 1) & 1u;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(bars + 32 + 8 * b, ph, a.status));
      tc_fence_after();
      const int r = (tile0 + tl) * 128 + r_in;
#pragma unroll
      for (int h = 0; h < NC; ++h) {
        // columns h * 2 MOUT .. + 2 MOUT: real parts, then imaginary parts, of set h
        constexpr int NW = ((2 * MOUT + 15) / 16) * 16;
        float v[NW];
#pragma unroll
        for (int c0 = 0; c0 < NW; c0 += 16)
          tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * 128 + h * 2 * MOUT + c0), v + c0);
        if (ok && r < a.n3) {
          float2* dst = a.out[h][t] + (long long)k * a.out_kstride + r;
#pragma unroll
          for (int j = 0; j < MOUT; ++j)
            if (j < a.mout) dst[(long long)j * a.n3] = make_float2(v[j], v[MOUT + j]);
        }
      }
      tc_fence_before();
      mbar_arrive(bars + 48 + 8 * b);
      if (!ok) break;
    }
  } else if (lane == 0) {
    const uint32_t idesc = idesc_bf16_n(NP);
    bool ok = true;
    for (int it = 0; it < nstage && ok; ++it) {
      const int s = it & 1;
      const uint32_t ph = (uint32_t)(it >> 1) & 1u;
      const int tl = it / nat, at = it % nat;
      const int b = tl & 1;
      if (at == 0) {  // accumulator buffer b must have been drained (use tl / 2 - 1)
        ok = mbar_wait(bars + 48 + 8 * b, ((uint32_t)(tl >> 1) & 1u) ^ 1u, a.status);
        if (!ok) break;
      }
      ok = mbar_wait(bars + 8 * s, ph, a.status);
      if (!ok) break;
      tc_fence_after();
      const uint32_t st = stg + s * U_STAGE;
      const uint64_t ah = sw128_desc(st), am = sw128_desc(st + A_SLICE), al = sw128_desc(st + 2 * A_SLICE);
      const uint64_t bh = sw128_desc(bop + (uint32_t)((0 * nat + at) * NP * 128));
      const uint64_t bm = sw128_desc(bop + (uint32_t)((1 * nat + at) * NP * 128));
      const uint64_t bl = sw128_desc(bop + (uint32_t)((2 * nat + at) * NP * 128));
      const uint32_t d = tmem + (uint32_t)(b * 128);
      const int nkk = min(4, (Kt - 64 * at + 15) / 16);
      for (int kk = 0; kk < nkk; ++kk) {
        const uint64_t off = (uint64_t)(2 * kk);
        mma_bf16(d, ah + off, bh + off, idesc, (at > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(d, ah + off, bm + off, idesc, 1u);
        mma_bf16(d, am + off, bh + off, idesc, 1u);
        mma_bf16(d, ah + off, bl + off, idesc, 1u);
        mma_bf16(d, am + off, bm + off, idesc, 1u);
        mma_bf16(d, al + off, bh + off, idesc, 1u);
      }
      mma_commit(bars + 16 + 8 * s);
      if (at == nat - 1) mma_commit(bars + 32 + 8 * b);
    }
    mma_commit(bars + 64);
    mbar_wait(bars + 64, 0u, a.status);  // every MMA of this CTA has completed
  }
  tc_fence_before();
  __syncthreads();
  if (warp == U_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
  }
}

template <int MOUT, int NC>
void set_update_smem() {
  // Once per instantiation; static initialisation is thread-safe (k groups run on several host threads).
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_tc_update<MOUT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, U_SMEM);
  (void)attr;
}

}  // namespace

// Split-reduction of the partial Gram matrices (defined with the CUDA-core kernels).
int launch_gram_reduce_f(const float2* part, int nsplit, int nel, int nk, float scale, float2* G, cudaStream_t s);

int launch_gram_tc(const float2* const A[3], int na, const float2* const B[3], int nbk, int nk, int m, int n3,
                   float scale, float2* part, int max_split, float2* G, int* status, cudaStream_t s) {
  if (na * m > 72 || nbk * m > 72 || nk < 1) return PC_EINVAL;
  static const cudaError_t attr =  // once, thread-safe static initialisation
      cudaFuncSetAttribute(k_tc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
  if (attr != cudaSuccess) {
    cudaGetLastError();
    return PC_ECUDA;
  }
  const int S = (n3 + 31) / 32;
  int ns = best_split(nk, S, max_split);
  const int per = (S + ns - 1) / ns;
  ns = (S + per - 1) / per;
  TcGramArgs a;
  for (int i = 0; i < 3; ++i) { a.A[i] = A[i]; a.B[i] = B[i]; }
  a.na = na; a.nbk = nbk; a.m = m; a.n3 = n3;
  a.nsplit = ns;
  a.rows_per_split = 32 * per;
  a.part = part;
  a.status = status;
  k_tc_gram<<<dim3(nk, ns), G_THREADS, G_SMEM, s>>>(a);
  PC_LAUNCH_CHECK();
  return launch_gram_reduce_f(part, ns, na * m * nbk * m, nk, scale, G, s);
}

int launch_update_tc(const UpdateArgs<float>& u, int* status, cudaStream_t s) {
  const int nc = u.C2nd ? 2 : 1;
  if (u.nblk * u.m > 72 || u.mout > 24 || u.mout < 1 || u.ntrip < 1 || u.ntrip > 3) return PC_EINVAL;
  TcUpdateArgs a;
  for (int t = 0; t < 3; ++t) {
    for (int b = 0; b < 3; ++b) a.in[t][b] = u.in[t][b];
    a.out[0][t] = u.out[t];
    a.out[1][t] = u.out2[t];
  }
  a.C[0] = u.C;
  a.C[1] = u.C2nd;
  a.cstride = u.cstride;
  a.cld = u.cld;
  a.nblk = u.nblk;
  a.identity_last = u.identity_last;
  a.m = u.m;
  a.mout = u.mout;
  a.n3 = u.n3;
  a.in_kstride = u.in_kstride;
  a.out_kstride = u.out_kstride;
  a.tiles = (u.n3 + 127) / 128;
  const int parts = best_split(u.nk * u.ntrip, a.tiles, 8);
  a.tiles_per_cta = (a.tiles + parts - 1) / parts;
  const int nz = (a.tiles + a.tiles_per_cta - 1) / a.tiles_per_cta;
  a.status = status;
  dim3 grid(u.nk, u.ntrip, nz);
  const int mo = u.mout <= 8 ? 8 : (u.mout <= 16 ? 16 : 24);
#define PC_TCU(MO, NCC)                                               \
  do {                                                                \
    set_update_smem<MO, NCC>();                                       \
    k_tc_update<MO, NCC><<<grid, U_THREADS, U_SMEM, s>>>(a);          \
  } while (0)
  if (nc == 1) {
    if (mo == 8) PC_TCU(8, 1); else if (mo == 16) PC_TCU(16, 1); else PC_TCU(24, 1);
  } else {
    if (mo == 8) PC_TCU(8, 2); else if (mo == 16) PC_TCU(16, 2); else PC_TCU(24, 2);
  }
#undef PC_TCU
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// ---------------------------------------------------------------------------
// Self-check of the tensor-core kernels against the CUDA-core kernels on seeded data.
namespace {
// A wait that cannot complete: no thread arrives on the barrier, so the bounded wait used by
// every tensor-core kernel must give up after `limit` polls, record PC_ETIMEOUT and return.
__global__ void k_wait_expiry(int* status, long long limit) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(b, 0u, status, limit);
}

__global__ void k_fill_hash(float2* p, long long n, unsigned long long seed, int n3) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto h = [](unsigned long long x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
    return x;
  };
  unsigned long long a = h(seed * 0x9e3779b97f4a7c15ull + (unsigned long long)i);
  // columns of very different norms, as in a block of search directions
  const float col_scale = exp2f((float)((i / n3) % 7) - 3.f);
  float re = ((float)(a & 0xffffff) / 16777216.f - 0.5f) * col_scale;
  float im = ((float)((a >> 24) & 0xffffff) / 16777216.f - 0.5f) * col_scale;
  p[i] = make_float2(re, im);
}
double max_abs_diff(const float2* a, const float2* b, long long n, double* ref_max) {
  std::vector<float2> x(n), y(n);
  cudaMemcpy(x.data(), a, n * sizeof(float2), cudaMemcpyDeviceToHost);
  cudaMemcpy(y.data(), b, n * sizeof(float2), cudaMemcpyDeviceToHost);
  double d = 0, r = 0;
  for (long long i = 0; i < n; ++i) {
    d = fmax(d, fmax(fabs((double)x[i].x - y[i].x), fabs((double)x[i].y - y[i].y)));
    r = fmax(r, fmax(fabs((double)y[i].x), fabs((double)y[i].y)));
  }
  *ref_max = r;
  return d;
}
}  // namespace

extern "C" int pc_check_tensor_kernels(int what, int nk, int m, int nblk, int n3, double* rel_err) {
  if (!rel_err) return PC_EINVAL;
  if (what == 2) {  // failure path of the bounded waits
    *rel_err = -1.0;
    int* st = nullptr;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) return PC_ENOMEM;
    int h = -1;
    bool ok = cudaMemset(st, 0, sizeof(int)) == cudaSuccess;
    k_wait_expiry<<<1, 32>>>(st, 1 << 14);
    ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    ok = ok && cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    // the context must still take work after the expired wait
    ok = ok && cudaMemset(st, 0, sizeof(int)) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    cudaFree(st);
    if (!ok) { cudaGetLastError(); return PC_ECUDA; }
    *rel_err = (h == PC_ETIMEOUT) ? 0.0 : 1.0;
    return PC_OK;
  }
  if (what == 3) return oz_self_check(n3, nk * m, rel_err);  // n3: plane waves, nk * m columns
  if (nk < 1 || m < 1 || m > 24 || nblk < 1 || nblk > 3 || n3 < 1 || (what != 0 && what != 1)) return PC_EINVAL;
  *rel_err = -1.0;
  const long long blk = (long long)nk * m * n3;
  float2 *in = nullptr, *out_tc = nullptr, *out_ref = nullptr, *C = nullptr, *part = nullptr;
  int* status = nullptr;
  const long long cel = (long long)nk * 72 * 72;
  bool ok = cudaMalloc(&in, 9 * blk * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&out_tc, 6 * blk * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&out_ref, 6 * blk * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&C, 2 * cel * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&part, 8 * cel * sizeof(float2)) == cudaSuccess && cudaMalloc(&status, sizeof(int)) == cudaSuccess;
  int rc = PC_OK;
  if (!ok) rc = PC_ENOMEM;
  if (!rc) {
    cudaMemset(status, 0, sizeof(int));
    k_fill_hash<<<cdiv(9 * blk, 256), 256>>>(in, 9 * blk, 1234567ull + what, n3);
    k_fill_hash<<<cdiv(2 * cel, 256), 256>>>(C, 2 * cel, 7654321ull, 1 << 30);
    cudaMemset(out_tc, 0, 6 * blk * sizeof(float2));
    cudaMemset(out_ref, 0, 6 * blk * sizeof(float2));
    const int saved = g_tc_tall;
    double d = 0, r = 0;
    if (what == 0) {
      // G = [in_0 .. in_{nblk-1}]^H [in_3 .. in_{3+nblk-1}], scale 1
      BlockList<float> A = {{in, in + blk, in + 2 * blk}}, B = {{in + 3 * blk, in + 4 * blk, in + 5 * blk}};
      g_tc_tall = 1;
      rc = launch_gram<float>(A, nblk, B, nblk, nk, m, n3, 1.f, part, out_tc, 0, status);
      g_tc_tall = 0;
      if (!rc) rc = launch_gram<float>(A, nblk, B, nblk, nk, m, n3, 1.f, part, out_ref, 0, nullptr);
      cudaDeviceSynchronize();
      if (!rc) d = max_abs_diff(out_tc, out_ref, (long long)nk * nblk * m * nblk * m, &r);
    } else {
      // three triplets, two coefficient sets, last block identity when nblk > 1
      UpdateArgs<float> u;
      memset(&u, 0, sizeof(u));
      for (int t = 0; t < 3; ++t) {
        for (int b = 0; b < nblk; ++b) u.in[t][b] = in + (3 * t + b) * blk;
        u.out[t] = out_tc + t * blk;
        u.out2[t] = out_tc + (3 + t) * blk;
      }
      u.ntrip = 3;
      u.nblk = nblk;
      u.identity_last = nblk > 1 ? 1 : 0;
      u.C = C;
      u.C2nd = C + cel;
      u.cstride = 72 * 72;
      u.cld = 72;
      u.m = m;
      u.mout = m;
      u.n3 = n3;
      u.nk = nk;
      u.in_kstride = (long long)m * n3;
      u.out_kstride = (long long)m * n3;
      u.status = status;
      g_tc_tall = 1;
      rc = launch_update<float>(u, 0);
      UpdateArgs<float> v = u;
      for (int t = 0; t < 3; ++t) { v.out[t] = out_ref + t * blk; v.out2[t] = out_ref + (3 + t) * blk; }
      v.status = nullptr;
      g_tc_tall = 0;
      if (!rc) rc = launch_update<float>(v, 0);
      cudaDeviceSynchronize();
      if (!rc) d = max_abs_diff(out_tc, out_ref, 6 * blk, &r);
    }
    g_tc_tall = saved;
    int st = 0;
    cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = PC_ECUDA;
    if (!rc && st) rc = st;
    if (!rc) *rel_err = r > 0 ? d / r : d;
  }
  cudaFree(in); cudaFree(out_tc); cudaFree(out_ref); cudaFree(C); cudaFree(part); cudaFree(status);
  return rc;
}
