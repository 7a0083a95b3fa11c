// Batched block operations of the locally optimal block preconditioned conjugate
// gradient iteration (one independent problem per k-point), and the small projected
// problems solved one CTA per k:
//   gram   -- G = A^H B over the 3N rows, for up to three m-column blocks per side
//   update -- out = [S_0 S_1 S_2] C for up to three operand triplets sharing C
//   small_rr   -- the projected pencil (GA, GO): unit-diagonal scaling, Cholesky of GO that
//                 drops dependent columns, reduction to standard form, cyclic Jacobi,
//                 lowest m Ritz pairs
//   small_chol -- Cholesky-QR transform T with T^H G T = I (dependent columns -> zero)
#include <type_traits>
#include "kernels.h"
#include "small_dense.cuh"

#define GRAM_SPLIT 8
#define GRAM_LD 73   // odd row stride of the shared tiles (columns up to 72)


// G_part[k][split] = A^H B over one row range; each of the 16 x 16 threads holds TILE x TILE outputs.  Shared tiles are double-buffered: the next
// tile of GRAM_ROWS rows (16 in FP32, 8 in FP64: 37 KB of static shared memory either way)
// is fetched into registers while the current one is multiplied.
template <typename R, typename RA, int TILE>
__global__ __launch_bounds__(256) void k_gram(BlockList<R> A, int na, BlockList<R> B, int nbk, int m, int n3,
                                              typename cplx_t<R>::type* __restrict__ part) {
  typedef typename cplx_t<R>::type C2;
  typedef typename cplx_t<RA>::type CA;
  constexpr int GRAM_ROWS = sizeof(R) == 8 ? 8 : 16;
  __shared__ C2 sA[2][GRAM_ROWS * GRAM_LD];
  __shared__ C2 sB[2][GRAM_ROWS * GRAM_LD];
  const int k = blockIdx.x, split = blockIdx.y;
  const int ca = na * m, cb = nbk * m;
  const long long kofs = (long long)k * m * n3;
  const int chunk = (n3 + GRAM_SPLIT - 1) / GRAM_SPLIT;
  const int r_begin = split * chunk, r_end = min(n3, r_begin + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // each thread stages elements t = threadIdx.x + 256 u of the (rows x cols) tiles
  const int nla = (GRAM_ROWS * ca + 255) / 256, nlb = (GRAM_ROWS * cb + 255) / 256;  // <= 5 (<= 3 in FP64)
  C2 ra[5], rb[5];
  auto fetch = [&](int r0) {
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      int t = threadIdx.x + 256 * u;
      ra[u] = mk<R>(0, 0);
      rb[u] = mk<R>(0, 0);
      if (u < nla && t < GRAM_ROWS * ca) {
        int rr = t % GRAM_ROWS, col = t / GRAM_ROWS, r = r0 + rr;
        if (r < r_end) ra[u] = A.p[col / m][kofs + (long long)(col % m) * n3 + r];
      }
      if (u < nlb && t < GRAM_ROWS * cb) {
        int rr = t % GRAM_ROWS, col = t / GRAM_ROWS, r = r0 + rr;
        if (r < r_end) rb[u] = B.p[col / m][kofs + (long long)(col % m) * n3 + r];
      }
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      int t = threadIdx.x + 256 * u;
      if (u < nla && t < GRAM_ROWS * ca) sA[buf][(t % GRAM_ROWS) * GRAM_LD + t / GRAM_ROWS] = ra[u];
      if (u < nlb && t < GRAM_ROWS * cb) sB[buf][(t % GRAM_ROWS) * GRAM_LD + t / GRAM_ROWS] = rb[u];
    }
  };
  CA acc[TILE][TILE];
#pragma unroll
  for (int i = 0; i < TILE; ++i)
#pragma unroll
    for (int j = 0; j < TILE; ++j) acc[i][j] = mk<RA>(0, 0);
  int buf = 0;
  if (r_begin < r_end) {
    fetch(r_begin);
    stash(0);
  }
  __syncthreads();
  for (int r0 = r_begin; r0 < r_end; r0 += GRAM_ROWS) {
    const bool more = r0 + GRAM_ROWS < r_end;
    if (more) fetch(r0 + GRAM_ROWS);
    const C2* a_t = sA[buf];
    const C2* b_t = sB[buf];
#pragma unroll 4
    for (int rr = 0; rr < GRAM_ROWS; ++rr) {
      C2 a[TILE], b[TILE];
#pragma unroll
      for (int i = 0; i < TILE; ++i) { int c = tx + 16 * i; a[i] = c < ca ? a_t[rr * GRAM_LD + c] : mk<R>(0, 0); }
#pragma unroll
      for (int j = 0; j < TILE; ++j) { int c = ty + 16 * j; b[j] = c < cb ? b_t[rr * GRAM_LD + c] : mk<R>(0, 0); }
#pragma unroll
      for (int i = 0; i < TILE; ++i)
#pragma unroll
        for (int j = 0; j < TILE; ++j) cfmac(acc[i][j], mk<RA>(a[i].x, a[i].y), mk<RA>(b[j].x, b[j].y));
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  C2* out = part + ((long long)k * GRAM_SPLIT + split) * ca * cb;
#pragma unroll
  for (int i = 0; i < TILE; ++i)
#pragma unroll
    for (int j = 0; j < TILE; ++j) {
      int a_ = tx + 16 * i, b_ = ty + 16 * j;
      if (a_ < ca && b_ < cb) out[a_ * cb + b_] = mk<R>((R)acc[i][j].x, (R)acc[i][j].y);
    }
}

template <typename R>
__global__ void k_gram_reduce(const typename cplx_t<R>::type* __restrict__ part, int nsplit, int nel, R scale,
                              typename cplx_t<R>::type* __restrict__ G) {
  typedef typename cplx_t<R>::type C2;
  int k = blockIdx.y;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const C2* p = part + (long long)k * nsplit * nel + e;
  C2 s = mk<R>(0, 0);
  for (int i = 0; i < nsplit; ++i) s = cadd(s, p[(long long)i * nel]);
  G[(long long)k * nel + e] = cscale(s, scale);
}

int launch_gram_reduce_f(const float2* part, int nsplit, int nel, int nk, float scale, float2* G, cudaStream_t s) {
  dim3 g2(cdiv(nel, 256), nk);
  k_gram_reduce<float><<<g2, 256, 0, s>>>(part, nsplit, nel, scale, G);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

template <typename R>
int launch_gram(BlockList<R> A, int na, BlockList<R> B, int nbk, int nk, int m, int n3, R scale,
                typename cplx_t<R>::type* part, typename cplx_t<R>::type* G, cudaStream_t s, int* status) {
  if (na * m > 72 || nbk * m > 72 || na * m > 80) return PC_EINVAL;
  if constexpr (std::is_same<R, float>::value) {
    if (g_tc_tall && status) return launch_gram_tc(A.p, na, B.p, nbk, nk, m, n3, scale, part, GRAM_SPLIT, G, status, s);
  }
  dim3 grid(nk, GRAM_SPLIT);
  // 16 x 16 threads, TILE x TILE outputs each: 2 x 2 covers up to 32 columns per side
  const bool small = na * m <= 32 && nbk * m <= 32;
  if (small) k_gram<R, R, 2><<<grid, 256, 0, s>>>(A, na, B, nbk, m, n3, part);
  else k_gram<R, R, 5><<<grid, 256, 0, s>>>(A, na, B, nbk, m, n3, part);
  PC_LAUNCH_CHECK();
  int nel = na * m * nbk * m;
  dim3 g2(cdiv(nel, 256), nk);
  k_gram_reduce<R><<<g2, 256, 0, s>>>(part, GRAM_SPLIT, nel, scale, G);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
template int launch_gram<double>(BlockList<double>, int, BlockList<double>, int, int, int, int, double, double2*, double2*, cudaStream_t, int*);
template int launch_gram<float>(BlockList<float>, int, BlockList<float>, int, int, int, int, float, float2*, float2*, cudaStream_t, int*);

// ---------------------------------------------------------------------------
// out[t][k][j][r] = (identity_last ? in[t][last][k][j][r] : 0) + sum_b sum_i in[t][b][k][i][r] C[k][b*m+i][j]
// One thread per row r: every row of every output is written by the thread that read it,
// so the output may alias the last input block.
template <typename R, int MOUT, typename RA>
__global__ __launch_bounds__(128) void k_update(UpdateArgs<R> a) {
  typedef typename cplx_t<R>::type C2;
  typedef typename cplx_t<RA>::type CA;
  __shared__ C2 sC[72 * 24];
  const int k = blockIdx.y, t = blockIdx.z;
  const int nsum = a.identity_last ? a.nblk - 1 : a.nblk;
  const int rows = nsum * a.m;
  const C2* Ck = a.C + (long long)k * a.cstride;
  for (int e = threadIdx.x; e < rows * a.mout; e += blockDim.x) {
    int i = e / a.mout, j = e % a.mout;
    sC[e] = Ck[(long long)i * a.cld + j];
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n3) return;
  CA acc[MOUT];
#pragma unroll
  for (int j = 0; j < MOUT; ++j) acc[j] = mk<RA>(0, 0);
  if (a.identity_last) {
    const C2* src = a.in[t][a.nblk - 1] + (long long)k * a.in_kstride + r;
#pragma unroll
    for (int j = 0; j < MOUT; ++j)
      if (j < a.mout) { C2 v = src[(long long)j * a.n3]; acc[j] = mk<RA>(v.x, v.y); }
  }
  for (int b = 0; b < nsum; ++b) {
    const C2* src = a.in[t][b] + (long long)k * a.in_kstride + r;
    for (int i = 0; i < a.m; ++i) {
      C2 v = src[(long long)i * a.n3];
      CA va = mk<RA>(v.x, v.y);
      const C2* crow = sC + (b * a.m + i) * a.mout;
#pragma unroll
      for (int j = 0; j < MOUT; ++j)
        if (j < a.mout) cfma(acc[j], va, mk<RA>(crow[j].x, crow[j].y));
    }
  }
  C2* dst = a.out[t] + (long long)k * a.out_kstride + r;
#pragma unroll
  for (int j = 0; j < MOUT; ++j)
    if (j < a.mout) dst[(long long)j * a.n3] = mk<R>((R)acc[j].x, (R)acc[j].y);
}

template <typename R> static int launch_update_cuda(const UpdateArgs<R>& a, cudaStream_t s) {
  int nsum = a.identity_last ? a.nblk - 1 : a.nblk;
  if (nsum * a.m * a.mout > 72 * 24 || a.mout > 24) return PC_EINVAL;
  dim3 grid(cdiv(a.n3, 128), a.nk, a.ntrip);
  if (a.mout <= 8) k_update<R, 8, R><<<grid, 128, 0, s>>>(a);
  else if (a.mout <= 16) k_update<R, 16, R><<<grid, 128, 0, s>>>(a);
  else k_update<R, 24, R><<<grid, 128, 0, s>>>(a);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// out[t] = [in] C (and out2[t] = [in] C2nd when a second coefficient set is given).  The CUDA-core
// kernel takes one set per launch; the tensor-core kernel (FP32) takes both in one pass.
template <typename R> int launch_update(const UpdateArgs<R>& a, cudaStream_t s) {
  if constexpr (std::is_same<R, float>::value) {
    if (g_tc_tall && a.status) return launch_update_tc(a, a.status, s);
  }
  int rc = launch_update_cuda<R>(a, s);
  if (rc || !a.C2nd) return rc;
  UpdateArgs<R> b = a;
  b.C = a.C2nd;
  for (int t = 0; t < 3; ++t) b.out[t] = a.out2[t];
  b.C2nd = nullptr;
  return launch_update_cuda<R>(b, s);
}
template int launch_update<double>(const UpdateArgs<double>&, cudaStream_t);
template int launch_update<float>(const UpdateArgs<float>&, cudaStream_t);

// ---------------------------------------------------------------------------
// Small dense Hermitian algebra in shared memory, one CTA per problem.  Matrices are stored
// row-major with an odd leading dimension ld (n + 1 for even n) so that column-wise accesses
// of consecutive threads fall into distinct banks.
template <typename R> struct SmallEps;
template <> struct SmallEps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct SmallEps<float>  { static constexpr float v = 1.1920929e-07f; };

// Rotation of one Jacobi plane: s complex, c real, p | q << 16 packed (16 bytes in FP32).
template <typename R> struct __align__(16) JPlane {
  typename cplx_t<R>::type s;
  R c;
  int pq;
};

// Two-sided cyclic Jacobi on Hermitian A (n x n, stride ld), accumulating V <- V J.  Pairs
// are scheduled by the circle method so each round rotates n/2 disjoint planes in parallel.
// A pair is rotated when |a_pq| > eps sqrt(|a_pp a_qq|) + eps max_{i < nx} |a_ii|, where the
// first nx coordinates carry the current Ritz block: the absolute term is the rounding floor
// at the scale of the wanted eigenvalues (near-zero modes would otherwise keep rotating
// noise).  The iteration ends after the first sweep that rotates nothing (or max_sweeps).
//
// One round is one pass over A: the planes partition the index set, so A splits into 2 x 2
// blocks (plane t1 rows, plane t2 columns), and J^H A J maps each block to L_t1 M R_t2 on its
// own.  Only blocks with t1 <= t2 are computed (their list is built once); each writes its
// conjugate transpose to block (t2, t1), which keeps A exactly Hermitian.  The planes of the
// next round depend on A only, so they are computed (by npairs threads) while the other
// threads rotate the column pairs of V for the current round, JV_ROWS rows per thread; the
// plane parameters are double-buffered by round.
// Scratch: pl (2 x 64 planes), blk (npairs (npairs + 1) / 2 ints), red (2 blockDim).
#define JV_ROWS 8
template <typename R>
__device__ void jacobi(typename cplx_t<R>::type* A, typename cplx_t<R>::type* V, int n, int ld, int nx, int max_sweeps,
                       JPlane<R>* pl, int* blk, R* red, const int* drop) {
  typedef typename cplx_t<R>::type C2;
  __shared__ int rot[2];  // a rotation happened in the sweep (by sweep parity)
  const int npad = n + (n & 1);
  const int npairs = npad / 2;
  const int nrounds = npad - 1;
  const R eps = SmallEps<R>::v;
  // exact Hermitian start: the triangular reductions leave rounding-level asymmetry
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    if (j > i) {
      C2 u = A[i * ld + j], l = A[j * ld + i];
      C2 h = mk<R>((u.x + l.x) * (R)0.5, (u.y - l.y) * (R)0.5);
      A[i * ld + j] = h;
      A[j * ld + i] = cconj(h);
    } else if (j == i) {
      A[i * ld + i].y = 0;
    }
  }
  // upper block list (t1 <= t2), packed t1 | t2 << 8
  const int nA = npairs * (npairs + 1) / 2;
  for (int e = threadIdx.x; e < npairs * npairs; e += blockDim.x) {
    const int t1 = e / npairs, t2 = e % npairs;
    if (t1 <= t2) blk[t1 * npairs - t1 * (t1 - 1) / 2 + (t2 - t1)] = t1 | (t2 << 8);
  }
  R amax = 0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x)
    if (!drop[i]) amax = fmax(amax, fabs(A[i * ld + i].x));
  red[threadIdx.x] = amax;
  if (threadIdx.x == 0) { rot[0] = 0; rot[1] = 0; }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const R floor_abs = eps * red[0];
  const int nch = (n + JV_ROWS - 1) / JV_ROWS;
  const int nV = npairs * nch;
  // rotation of plane t in the given round, from the current A
  auto plane = [&](int round, int t, JPlane<R>* dst, int* flag) {
    int a = (t == 0) ? 0 : ((t - 1 + round) % nrounds) + 1;
    int b = ((nrounds - t - 1 + round) % nrounds) + 1;
    int p = min(a, b), q = max(a, b);
    R c = 1;
    C2 sp = mk<R>(0, 0);
    if (q < n && !drop[p] && !drop[q]) {
      C2 apq = A[p * ld + q];
      R beta = sqrt(apq.x * apq.x + apq.y * apq.y);
      R app = A[p * ld + p].x, aqq = A[q * ld + q].x;
      if (beta > eps * sqrt(fabs(app) * fabs(aqq)) + floor_abs) {
        R tau = (aqq - app) / (2 * beta);
        R tt = (tau >= 0 ? (R)1 : (R)-1) / (fabs(tau) + sqrt((R)1 + tau * tau));
        c = (R)1 / sqrt((R)1 + tt * tt);
        R sn = tt * c;
        sp = mk<R>(sn * apq.x / beta, sn * apq.y / beta);
        *flag = 1;
      }
    }
    JPlane<R> w;
    w.c = c;
    w.s = sp;
    w.pq = p | (q << 16);
    dst[t] = w;
  };
  for (int t = threadIdx.x; t < npairs; t += blockDim.x) plane(0, t, pl, &rot[0]);
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < nrounds; ++round) {
      const int g = sweep * nrounds + round;
      const JPlane<R>* cur = pl + (g & 1) * 64;
      JPlane<R>* nxt = pl + ((g + 1) & 1) * 64;
      // A <- J^H A J: block (t1, t2), rows p1, q1 and columns p2, q2
      for (int e = threadIdx.x; e < nA; e += blockDim.x) {
        const int tt12 = blk[e];
        const int t1 = tt12 & 255, t2 = tt12 >> 8;
        const JPlane<R> w1 = cur[t1], w2 = cur[t2];
        const C2 s1 = w1.s, s2 = w2.s;
        const bool a1 = (s1.x != 0 || s1.y != 0), a2 = (s2.x != 0 || s2.y != 0);
        if (!a1 && !a2) continue;
        const R c1 = w1.c, c2 = w2.c;
        const int p1 = w1.pq & 0xffff, q1 = w1.pq >> 16, p2 = w2.pq & 0xffff, q2 = w2.pq >> 16;
        const bool v1 = q1 < n, v2 = q2 < n;
        const C2 z = mk<R>(0, 0);
        C2 m00 = A[p1 * ld + p2];
        C2 m01 = v2 ? A[p1 * ld + q2] : z;
        C2 m10 = v1 ? A[q1 * ld + p2] : z;
        C2 m11 = (v1 && v2) ? A[q1 * ld + q2] : z;
        // columns (plane t2): col_p <- c col_p - conj(s) col_q, col_q <- s col_p + c col_q
        const C2 s2c = cconj(s2);
        C2 y00 = csub(cscale(m00, c2), cmul(s2c, m01)), y01 = cadd(cmul(s2, m00), cscale(m01, c2));
        C2 y10 = csub(cscale(m10, c2), cmul(s2c, m11)), y11 = cadd(cmul(s2, m10), cscale(m11, c2));
        // rows (plane t1): row_p <- c row_p - s row_q, row_q <- conj(s) row_p + c row_q
        const C2 s1c = cconj(s1);
        m00 = csub(cscale(y00, c1), cmul(s1, y10));
        m01 = csub(cscale(y01, c1), cmul(s1, y11));
        m10 = cadd(cmul(s1c, y00), cscale(y10, c1));
        m11 = cadd(cmul(s1c, y01), cscale(y11, c1));
        if (t1 == t2) {  // the rotated plane itself: its off-diagonal pair is annihilated
          A[p1 * ld + p1] = mk<R>(m00.x, 0);
          if (v1) {
            A[q1 * ld + q1] = mk<R>(m11.x, 0);
            A[p1 * ld + q1] = z;
            A[q1 * ld + p1] = z;
          }
        } else {
          A[p1 * ld + p2] = m00;
          A[p2 * ld + p1] = cconj(m00);
          if (v2) { A[p1 * ld + q2] = m01; A[q2 * ld + p1] = cconj(m01); }
          if (v1) { A[q1 * ld + p2] = m10; A[p2 * ld + q1] = cconj(m10); }
          if (v1 && v2) { A[q1 * ld + q2] = m11; A[q2 * ld + q1] = cconj(m11); }
        }
      }
      __syncthreads();
      // planes of the next round (the first npairs threads) while the others rotate V
      if ((int)threadIdx.x < npairs) {
        const bool last = round + 1 == nrounds;
        plane(last ? 0 : round + 1, threadIdx.x, nxt, &rot[(sweep + (last ? 1 : 0)) & 1]);
      } else {
        for (int e2 = threadIdx.x - npairs; e2 < nV; e2 += blockDim.x - npairs) {
          // rows c0, c0 + nch, c0 + 2 nch, ... of V, column pair of plane t: V <- V J
          // (neighbouring lanes take neighbouring rows: distinct banks with the odd stride)
          const int t = e2 / nch, c0 = e2 - t * nch;
          const JPlane<R> w = cur[t];
          const C2 sp = w.s;
          if (sp.x == 0 && sp.y == 0) continue;
          const int p = w.pq & 0xffff, q = w.pq >> 16;
          const R c = w.c;
          const C2 spc = cconj(sp);
#pragma unroll 4
          for (int i = c0; i < n; i += nch) {
            const C2 vip = V[i * ld + p], viq = V[i * ld + q];
            V[i * ld + p] = csub(cscale(vip, c), cmul(spc, viq));
            V[i * ld + q] = cadd(cmul(sp, vip), cscale(viq, c));
          }
        }
      }
      __syncthreads();
    }
    // sweep finished: stop if it rotated nothing (the planes already computed for the next
    // sweep came from an unchanged A and are dropped)
    const bool done = (rot[sweep & 1] == 0);
    __syncthreads();
    if (threadIdx.x == 0) rot[sweep & 1] = 0;  // reused by sweep + 2
    if (done) break;
  }
  __syncthreads();
}

#define SMALL_THREADS 1024
template <typename R> struct SmallSmem {
  static int ld(int n) { return n + ((n & 1) ? 0 : 1); }
  static size_t bytes(int n) {
    typedef typename cplx_t<R>::type C2;
    const int L = ld(n);
    return sizeof(C2) * (2 * (size_t)n * L + n) + sizeof(JPlane<R>) * 128 + sizeof(R) * (2 * n + 2 * SMALL_THREADS) +
           sizeof(int) * (2 * n + 64 * 65 / 2 + 16);
  }
};

template <typename R>
__global__ __launch_bounds__(SMALL_THREADS) void k_small_rr(const typename cplx_t<R>::type* __restrict__ GA,
                                                            const typename cplx_t<R>::type* __restrict__ GO, int n, int m,
                                                            R drop_tol, const int* __restrict__ kdone,
                                                            R* __restrict__ lam_out,
                                                            typename cplx_t<R>::type* __restrict__ coef, int* status) {
  typedef typename cplx_t<R>::type C2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ld = n + ((n & 1) ? 0 : 1);
  C2* A = (C2*)smem;                 // n*ld
  C2* B = A + n * ld;                // n*ld
  JPlane<R>* pl = (JPlane<R>*)(B + n * ld);  // 2 x 64 planes
  C2* tmp = (C2*)(pl + 128);         // n
  R* D = (R*)(tmp + n);              // n
  R* ev = D + n;                     // n
  R* red = ev + n;                   // 2 * SMALL_THREADS
  int* drop = (int*)(red + 2 * SMALL_THREADS);  // n
  int* perm = drop + n;              // n
  int* blk = perm + n;               // 64 * 65 / 2 upper blocks
  int* cnt = blk + 64 * 65 / 2;
  const int k = blockIdx.x;
  const C2* ga = GA + (long long)k * n * n;
  const C2* go = GO + (long long)k * n * n;
  if (kdone && kdone[k]) {  // locked k-point: keep its block, leave lambda untouched
    C2* ck = coef + (long long)k * n * m;
    for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
      int i = t / m, j = t % m;
      ck[t] = (i == j) ? mk<R>(1, 0) : mk<R>(0, 0);
    }
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    R d = go[i * n + i].x;
    D[i] = (d > (R)0 && d == d) ? (R)1 / sqrt(d) : (R)0;
    drop[i] = 0;
  }
  __syncthreads();
  // Hermitian-symmetrised, unit-diagonal-scaled copies
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, c = t % n;
    C2 a1 = ga[i * n + c], a2 = ga[c * n + i];
    C2 b1 = go[i * n + c], b2 = go[c * n + i];
    R s = D[i] * D[c] * (R)0.5;
    A[i * ld + c] = mk<R>((a1.x + a2.x) * s, (a1.y - a2.y) * s);
    B[i * ld + c] = mk<R>((b1.x + b2.x) * s, (b1.y - b2.y) * s);
  }
  __syncthreads();
  chol_drop<R>(B, n, ld, drop_tol, drop);
  tri_inv_lower<R>(B, n, ld, tmp);  // B = Li (lower)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // A <- A Li^H, one warp per row
  for (int i = warp; i < n; i += nw) {
    C2 outv[3];
    int cj = 0;
    for (int j = lane; j < n && cj < 3; j += 32, ++cj) {
      C2 s = mk<R>(0, 0);
      for (int c = 0; c <= j; ++c) cfmac(s, B[j * ld + c], A[i * ld + c]);  // sum_c A[i][c] conj(Li[j][c])
      outv[cj] = s;
    }
    __syncwarp();
    cj = 0;
    for (int j = lane; j < n && cj < 3; j += 32, ++cj) A[i * ld + j] = outv[cj];
    __syncwarp();
  }
  __syncthreads();
  // A <- Li A, one warp per column
  for (int j = warp; j < n; j += nw) {
    C2 outv[3];
    int ci = 0;
    for (int i = lane; i < n && ci < 3; i += 32, ++ci) {
      C2 s = mk<R>(0, 0);
      for (int c = 0; c <= i; ++c) cfma(s, B[i * ld + c], A[c * ld + j]);
      outv[ci] = s;
    }
    __syncwarp();
    ci = 0;
    for (int i = lane; i < n && ci < 3; i += 32, ++ci) A[i * ld + j] = outv[ci];
    __syncwarp();
  }
  __syncthreads();
  // dropped coordinates: decoupled; Jacobi leaves them alone and the sort puts them last
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, c = t % n;
    if (drop[i] || drop[c]) A[i * ld + c] = mk<R>(0, 0);
  }
  __syncthreads();
  // B <- Li^H (conjugate transpose in place): V starts as Li^H so that V J = Li^H Y
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, c = t % n;
    if (c > i) {
      C2 lo = B[c * ld + i];
      B[i * ld + c] = cconj(lo);
      B[c * ld + i] = mk<R>(0, 0);
    } else if (c == i) {
      B[i * ld + c] = cconj(B[i * ld + c]);
    }
  }
  __syncthreads();
  jacobi<R>(A, B, n, ld, m, 30, pl, blk, red, drop);
  for (int i = threadIdx.x; i < n; i += blockDim.x) ev[i] = A[i * ld + i].x;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int r = 0;
    R vi = ev[i];
    for (int j = 0; j < n; ++j) {
      bool before;
      if (drop[i] != drop[j]) before = drop[i] > drop[j];          // kept coordinates first
      else before = (ev[j] < vi || (ev[j] == vi && j < i));
      r += before ? 1 : 0;
    }
    perm[r] = i;
  }
  if (threadIdx.x == 0) {
    int kept = 0;
    for (int i = 0; i < n; ++i) kept += drop[i] ? 0 : 1;
    cnt[0] = kept;
  }
  __syncthreads();
  C2* ck = coef + (long long)k * n * m;
  if (cnt[0] < m) {
    // too few independent directions: keep the current block (identity on its first m coordinates)
    for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
      int i = t / m, j = t % m;
      ck[t] = (i == j) ? mk<R>(1, 0) : mk<R>(0, 0);
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) lam_out[(long long)k * m + j] = ga[j * n + j].x / go[j * n + j].x;
    if (threadIdx.x == 0) set_status(status, PC_ENOCONV);
    return;
  }
  for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
    int i = t / m, j = t % m;
    ck[t] = cscale(B[i * ld + perm[j]], D[i]);
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) lam_out[(long long)k * m + j] = ev[perm[j]];
}

template <typename R>
int launch_small_rr(const typename cplx_t<R>::type* GA, const typename cplx_t<R>::type* GO, int n, int m, int nk,
                    R drop_tol, const int* kdone, R* lam_out, typename cplx_t<R>::type* coef, int* status,
                    cudaStream_t s) {
  size_t sm = SmallSmem<R>::bytes(n);
  // Once per instantiation (thread-safe static initialisation: k groups run on several host threads).
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_small_rr<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  (void)attr;
  if (sm > 200 * 1024) return PC_EINVAL;
  k_small_rr<R><<<nk, SMALL_THREADS, sm, s>>>(GA, GO, n, m, drop_tol, kdone, lam_out, coef, status);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
template int launch_small_rr<double>(const double2*, const double2*, int, int, int, double, const int*, double*, double2*, int*, cudaStream_t);

// Cholesky-QR transform: T = D Li^H with zero columns for dropped coordinates.
template <typename R>
__global__ __launch_bounds__(256) void k_small_chol(const typename cplx_t<R>::type* __restrict__ G, int m, R drop_tol,
                                                    const typename cplx_t<R>::type* __restrict__ Gref, int rows_ref,
                                                    R rel_tol, typename cplx_t<R>::type* __restrict__ T) {
  typedef typename cplx_t<R>::type C2;
  __shared__ C2 B[24 * 25];
  __shared__ C2 tmp[24];
  __shared__ R D[24];
  __shared__ int drop[24];
  const int ld = m + ((m & 1) ? 0 : 1);
  const int k = blockIdx.x;
  const C2* g = G + (long long)k * m * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    R d = g[i * m + i].x;
    bool keep = (d > (R)0 && d == d);
    if (keep && Gref) {
      R before = -Gref[(long long)k * rows_ref * m + (long long)(rows_ref - m + i) * m + i].x;
      keep = d > rel_tol * before;
    }
    D[i] = keep ? (R)1 / sqrt(d) : (R)0;
    drop[i] = 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, c = t % m;
    C2 b1 = g[i * m + c], b2 = g[c * m + i];
    R s = D[i] * D[c] * (R)0.5;
    B[i * ld + c] = mk<R>((b1.x + b2.x) * s, (b1.y - b2.y) * s);
  }
  __syncthreads();
  chol_drop<R>(B, m, ld, drop_tol, drop);
  tri_inv_lower<R>(B, m, ld, tmp);
  C2* tk = T + (long long)k * m * m;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, c = t % m;
    // T[i][c] = D_i conj(Li[c][i]); dropped columns vanish
    C2 v = (c >= i && !drop[c]) ? cscale(cconj(B[c * ld + i]), D[i]) : mk<R>(0, 0);
    tk[t] = v;
  }
}
template <typename R>
int launch_small_chol(const typename cplx_t<R>::type* G, int m, int nk, R drop_tol,
                      const typename cplx_t<R>::type* Gref, int rows_ref, R rel_tol, typename cplx_t<R>::type* T,
                      cudaStream_t s) {
  if (m > 24) return PC_EINVAL;
  k_small_chol<R><<<nk, 256, 0, s>>>(G, m, drop_tol, Gref, rows_ref, rel_tol, T);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
template int launch_small_chol<double>(const double2*, int, int, double, const double2*, int, double, double2*, cudaStream_t);
template int launch_small_chol<float>(const float2*, int, int, float, const float2*, int, float, float2*, cudaStream_t);

// ---------------------------------------------------------------------------
// Conjugate-direction coefficients in the small space.  With the Ritz coefficients cX
// (cX^H GO cX = I) of the basis S = [X_old, W, P_old], the next conjugate block spans the
// part of span(X_old) that is GO-orthogonal to the new Ritz block:
//     Z = E - cX (cX^H GO E),  E = [I_m; 0],
// orthonormalised in the GO metric (H = Z^H GO Z, Cholesky-QR; columns with H_jj below
// abs_drop carry only rounding and are dropped).  span(X_new, P_new) = span(X_new, X_old),
// and P_new = S cP is formed from GO-orthonormal coefficients, so no cancellation is
// amplified in the tall update.  Locked k-points get cP = 0.
template <typename R>
__global__ __launch_bounds__(256) void k_small_pdir(const typename cplx_t<R>::type* __restrict__ GO,
                                                    const typename cplx_t<R>::type* __restrict__ CX, int n, int m,
                                                    const int* __restrict__ kdone, R abs_drop,
                                                    typename cplx_t<R>::type* __restrict__ CP) {
  typedef typename cplx_t<R>::type C2;
  extern __shared__ __align__(16) unsigned char smem[];
  C2* cx = (C2*)smem;         // n*m
  C2* z = cx + n * m;         // n*m
  C2* gz = z + n * m;         // n*m
  C2* Mm = gz + n * m;        // m*m  (also H, then T workspace)
  C2* tmp = Mm + m * m;       // m
  R* D = (R*)(tmp + m);       // m
  int* drop = (int*)(D + m);  // m
  const int k = blockIdx.x;
  C2* cp = CP + (long long)k * n * m;
  if (kdone && kdone[k]) {
    for (int t = threadIdx.x; t < n * m; t += blockDim.x) cp[t] = mk<R>(0, 0);
    return;
  }
  const C2* go = GO + (long long)k * n * n;
  const C2* cxg = CX + (long long)k * n * m;
  for (int t = threadIdx.x; t < n * m; t += blockDim.x) cx[t] = cxg[t];
  __syncthreads();
  // M = cX^H GO E  (GO symmetrised on the fly)
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, j = t % m;
    C2 s = mk<R>(0, 0);
    for (int r = 0; r < n; ++r) {
      C2 g1 = go[r * n + j], g2 = go[j * n + r];
      C2 g = mk<R>((R)0.5 * (g1.x + g2.x), (R)0.5 * (g1.y - g2.y));
      cfmac(s, cx[r * m + i], g);
    }
    Mm[t] = s;
  }
  __syncthreads();
  // Z = E - cX M
  for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
    int r = t / m, j = t % m;
    C2 s = mk<R>((r == j) ? (R)1 : (R)0, 0);
    for (int i = 0; i < m; ++i) {
      C2 v = cmul(cx[r * m + i], Mm[i * m + j]);
      s.x -= v.x; s.y -= v.y;
    }
    z[t] = s;
  }
  __syncthreads();
  // GZ = GO Z
  for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
    int r = t / m, j = t % m;
    C2 s = mk<R>(0, 0);
    for (int q = 0; q < n; ++q) {
      C2 g1 = go[r * n + q], g2 = go[q * n + r];
      C2 g = mk<R>((R)0.5 * (g1.x + g2.x), (R)0.5 * (g1.y - g2.y));
      cfma(s, g, z[q * m + j]);
    }
    gz[t] = s;
  }
  __syncthreads();
  // H = Z^H GZ, unit-diagonal scaled, dropped columns (H_jj <= abs_drop) decoupled
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    C2 s = mk<R>(0, 0);
    for (int r = 0; r < n; ++r) cfmac(s, z[r * m + i], gz[r * m + i]);
    D[i] = (s.x > abs_drop && s.x == s.x) ? (R)1 / sqrt(s.x) : (R)0;
    drop[i] = 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, j = t % m;
    C2 s1 = mk<R>(0, 0), s2 = mk<R>(0, 0);
    for (int r = 0; r < n; ++r) { cfmac(s1, z[r * m + i], gz[r * m + j]); cfmac(s2, z[r * m + j], gz[r * m + i]); }
    R sc = D[i] * D[j] * (R)0.5;
    Mm[t] = mk<R>((s1.x + s2.x) * sc, (s1.y - s2.y) * sc);
  }
  __syncthreads();
  chol_drop<R>(Mm, m, m, (R)1e-10, drop);
  tri_inv_lower<R>(Mm, m, m, tmp);
  // cP = Z T with T[i][c] = D_i conj(Li[c][i]) for c >= i and c kept
  for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
    int r = t / m, c = t % m;
    C2 s = mk<R>(0, 0);
    if (!drop[c] && D[c] != (R)0) {
      for (int i = 0; i <= c; ++i) {
        C2 tv = cscale(cconj(Mm[c * m + i]), D[i]);
        cfma(s, z[r * m + i], tv);
      }
    }
    cp[t] = s;
  }
}

template <typename R>
int launch_small_pdir(const typename cplx_t<R>::type* GO, const typename cplx_t<R>::type* CX, int n, int m, int nk,
                      const int* kdone, R abs_drop, typename cplx_t<R>::type* CP, cudaStream_t s) {
  typedef typename cplx_t<R>::type C2;
  if (m > 24 || n > 72) return PC_EINVAL;
  size_t sm = sizeof(C2) * (3 * (size_t)n * m + (size_t)m * m + m) + sizeof(R) * m + sizeof(int) * m + 64;
  static const cudaError_t attr =  // once per instantiation, thread-safe
      cudaFuncSetAttribute(k_small_pdir<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  (void)attr;
  k_small_pdir<R><<<nk, 256, sm, s>>>(GO, CX, n, m, kdone, abs_drop, CP);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
template int launch_small_pdir<double>(const double2*, const double2*, int, int, int, const int*, double, double2*, cudaStream_t);
template int launch_small_pdir<float>(const float2*, const float2*, int, int, int, const int*, float, float2*, cudaStream_t);
