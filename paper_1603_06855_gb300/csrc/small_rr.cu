// Projected Rayleigh-Ritz problems of the FP32 block iteration: one CTA per k-point solves the
// Hermitian pencil (GA, GO) of the basis S = [X W P] (n <= 72 columns) for its lowest m
// eigenpairs, with eigenvalues accurate relative to their own size.
//
// Steps (per k):
//  1. unit-diagonal scaling D = diag(GO)^-1/2 and Hermitian symmetrisation of both matrices;
//  2. Cholesky GO = L L^H, blocked: 8-column panels factored by one warp, then the trailing
//     update by all threads.  A pivot at or below drop_tol drops its coordinate (its row and
//     column of L become e_j);
//  3. T = L^-1 GA and L^-1, then C = L^-1 T^H = L^-1 GA L^-H, by blocked forward substitution
//     (8-row blocks: the update from the solved rows by all threads, then the 8 x 8 diagonal
//     solve one thread per column); V = L^-H is kept transposed (V^T = conj(L^-1));
//  4. the kept coordinates are packed into a position-ordered upper-triangular copy of C and
//     diagonalised by cyclic two-sided Jacobi, the n_k/2 disjoint planes of a round ordered
//     by the circle method.  Positions are pair-ordered: the planes of every round are the
//     position pairs (2t, 2t+1), and the rotated matrix is written to the other buffer at
//     the positions the next round gives its indices, so every 2 x 2 block is read from
//     adjacent rows and columns (16-byte loads).  The planes of the next round are computed
//     in the same pass from the entries they need (recomputed with the same arithmetic as
//     the block updates), so a round costs one barrier; blocks, planes and the updates of
//     V^T (two rows of two elements per unit, on the original coordinates) form one work list
//     shared by all threads.  A plane rotates when |a_uv| > eps sqrt(|a_uu a_vv|) +
//     eps max_{i < m} |a_ii| (the absolute floor is the rounding level of the current Ritz
//     block); after each sweep one pass over all pairs ends the iteration when none would
//     rotate.
//  5. the lowest m eigenvalues of the kept coordinates and their coefficients D V;
//  6. when asked, the conjugate-direction coefficients of the next iteration from the same
//     CTA (pdir32: Cholesky-QR of the part of the old Ritz block outside the new one).
// This is the mixed form's version (FP32, four 72 x 74 complex matrices in shared memory);
// the FP64 form keeps the kernel in lobpcg.cu.
#include "kernels.h"
#include "small_dense.cuh"

namespace {

constexpr int SR_THREADS = 1024;
constexpr int SR_NMAX = 72;
constexpr int SR_LD = 74;                       // even row stride: 16-byte aligned element pairs
constexpr int SR_MAT = SR_NMAX * SR_LD;         // complex elements per matrix
constexpr int SR_MAX_SWEEPS = 30;
constexpr int SR_BLK = 36 * 37 / 2;             // upper 2 x 2 blocks of 36 planes
constexpr int SR_PB = 8;                        // panel / row-block width of the reductions

// Complex arithmetic with explicit roundings, so that every call site computes bitwise the
// same value from the same inputs (the plane threads recompute entries the block threads
// store).
__device__ __forceinline__ float2 zmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 zconj(float2 a) { return make_float2(a.x, -a.y); }
// c x + z (c real)
__device__ __forceinline__ float2 zaxpy(float c, float2 x, float2 z) {
  return make_float2(__fmaf_rn(c, x.x, z.x), __fmaf_rn(c, x.y, z.y));
}
__device__ __forceinline__ float2 zneg(float2 a) { return make_float2(-a.x, -a.y); }

struct __align__(16) Plane {
  float2 s;  // rotation: col_u <- c col_u - conj(s) col_v, col_v <- s col_u + c col_v
  float c;
  int on;    // rotates (s != 0)
};

// Column part of the two-sided rotation of a 2 x 2 block M (rows: plane 1, columns: plane 2):
// y_a = (J2 applied to row a of M)[col].
__device__ __forceinline__ float2 col_rot(float2 ma0, float2 ma1, const Plane& p2, int col) {
  return col == 0 ? zaxpy(p2.c, ma0, zneg(zmul(zconj(p2.s), ma1))) : zaxpy(p2.c, ma1, zmul(p2.s, ma0));
}
// Row part: entry (row, col) of J1^H Y from the column-rotated pair (y0, y1) of that column.
__device__ __forceinline__ float2 row_rot(float2 y0, float2 y1, const Plane& p1, int row) {
  return row == 0 ? zaxpy(p1.c, y0, zneg(zmul(p1.s, y1))) : zaxpy(p1.c, y1, zmul(zconj(p1.s), y0));
}

// Next position of the circle method in pair-ordered positions (top[t] = 2t, bottom[t] = 2t+1):
// top[0] stays, top[t] -> top[t+1], top[np-1] -> bottom[np-1], bottom[t] -> bottom[t-1],
// bottom[0] -> top[1].  One cycle through the 2 np - 1 moving positions.
__device__ __forceinline__ int next_pos(int pos, int np) {
  if (np == 1 || pos == 0) return pos;
  if (pos & 1) return pos == 1 ? 2 : pos - 2;
  return (pos >> 1) == np - 1 ? pos + 1 : pos + 2;
}
__device__ __forceinline__ int prev_pos(int pos, int np) {
  if (np == 1 || pos == 0) return pos;
  if (pos & 1) return pos == 2 * np - 1 ? pos - 1 : pos + 2;
  return pos == 2 ? 1 : pos - 2;
}

// Upper-stored element (i, j) of a position-ordered Hermitian matrix.
__device__ __forceinline__ float2 uget(const float2* S, int i, int j) {
  return i <= j ? S[i * SR_LD + j] : zconj(S[j * SR_LD + i]);
}

// Entry (u, v) (positions, any order) of J^H A J for the planes pl of the current round.
__device__ __forceinline__ float2 rotated_entry(const float2* S, const Plane* pl, int u, int v) {
  int tu = u >> 1, tv = v >> 1, r = u & 1, c = v & 1;
  bool tr = false;
  if (tu > tv) { int t = tu; tu = tv; tv = t; t = r; r = c; c = t; tr = true; }
  const Plane p1 = pl[tu], p2 = pl[tv];
  if (tu == tv && p1.on && r != c) return make_float2(0.f, 0.f);  // annihilated by its own plane
  const int a0 = 2 * tu, b0 = 2 * tv;
  const float2 m00 = uget(S, a0, b0), m01 = uget(S, a0, b0 + 1), m10 = uget(S, a0 + 1, b0),
               m11 = uget(S, a0 + 1, b0 + 1);
  const float2 y0 = col_rot(m00, m01, p2, c), y1 = col_rot(m10, m11, p2, c);
  float2 e = row_rot(y0, y1, p1, r);
  if (tu == tv && r == c) e.y = 0.f;
  return tr ? zconj(e) : e;
}

// Rotation of the plane of positions (u, v) from a_uu, a_vv (real) and a_uv:
// with d = a_vv - a_uu and b = |a_uv|, t = 2 b sgn(d) / (|d| + sqrt(d^2 + 4 b^2)) is the tangent
// of the smaller rotation angle, c = 1 / sqrt(1 + t^2) and s = c t a_uv / b.
__device__ __forceinline__ Plane make_plane(float app, float aqq, float2 apq, float floor_abs, bool valid) {
  Plane w;
  w.c = 1.f;
  w.s = make_float2(0.f, 0.f);
  w.on = 0;
  const float eps = 1.1920929e-07f;
  const float b2 = apq.x * apq.x + apq.y * apq.y;
  const float b = __fsqrt_rn(b2);
  if (valid && b > eps * __fsqrt_rn(fabsf(app) * fabsf(aqq)) + floor_abs) {
    const float d = aqq - app;
    const float sg = d >= 0.f ? 1.f : -1.f;
    const float inv = __frcp_rn(fabsf(d) + __fsqrt_rn(d * d + 4.f * b2));
    const float t = 2.f * b * inv;                  // |tangent|
    const float c = __frsqrt_rn(1.f + t * t);
    const float f = 2.f * sg * inv * c;             // c t / b
    w.c = c;
    w.s = make_float2(f * apq.x, f * apq.y);
    w.on = 1;
  }
  return w;
}

// Forward substitution L X = R in place for ncol columns (column c of R is column c of P[0] for
// c < n0, else column c - n0 of P[1]); L lower with row stride SR_LD, drops already turned into
// e_j.  8-row blocks: the update of the block's rows from the rows solved before it (all
// threads, one output each), then the 8 x 8 diagonal solve (one thread per column).
__device__ __forceinline__ void block_forward(const float2* L, float2* const P[2], int n0, int n, int ncol) {
  const int tid = threadIdx.x;
  for (int i0 = 0; i0 < n; i0 += SR_PB) {
    const int ib = min(SR_PB, n - i0);
    if (i0 > 0) {
      for (int e = tid; e < ib * ncol; e += SR_THREADS) {
        const int ii = e / ncol, c = e - ii * ncol;
        float2* R = c < n0 ? P[0] + c : P[1] + (c - n0);
        const float2* Li = L + (i0 + ii) * SR_LD;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        int k = 0;
        for (; k + 1 < i0; k += 2) {
          cfma(a0, Li[k], R[k * SR_LD]);
          cfma(a1, Li[k + 1], R[(k + 1) * SR_LD]);
        }
        if (k < i0) cfma(a0, Li[k], R[k * SR_LD]);
        const float2 r = R[(i0 + ii) * SR_LD];
        R[(i0 + ii) * SR_LD] = make_float2(r.x - a0.x - a1.x, r.y - a0.y - a1.y);
      }
      __syncthreads();
    }
    for (int c = tid; c < ncol; c += SR_THREADS) {
      float2* R = c < n0 ? P[0] + c : P[1] + (c - n0);
      float2 x[SR_PB];
#pragma unroll
      for (int ii = 0; ii < SR_PB; ++ii) {
        if (ii < ib) {
          const int i = i0 + ii;
          float2 acc = R[i * SR_LD];
#pragma unroll
          for (int kk = 0; kk < ii; ++kk) {
            const float2 l = L[i * SR_LD + i0 + kk];
            acc.x -= l.x * x[kk].x - l.y * x[kk].y;
            acc.y -= l.x * x[kk].y + l.y * x[kk].x;
          }
          const float il = 1.f / L[i * SR_LD + i].x;
          x[ii] = make_float2(acc.x * il, acc.y * il);
          R[i * SR_LD] = x[ii];
        }
      }
    }
    __syncthreads();
  }
}

// Conjugate-direction coefficients, inside the CTA that solved the projected problem.  With the
// Ritz coefficients cX (n x m, cX^H GO cX = I) of the basis S = [X_old, W, P_old], the next
// conjugate block spans the part of span(X_old) that is GO-orthogonal to the new Ritz block:
// Z = E - cX (cX^H GO E), E = [I_m; 0], orthonormalised in the GO metric (H = Z^H GO Z,
// unit-diagonal scaled, Cholesky-QR; columns with H_jj at or below abs_drop carry only rounding
// and are dropped), cP = Z T.  go: the projected Gram matrix (global); G (stride SR_LD), cx, z, gz
// (n x m compact), Mm (m x m), tmp (m), Dd (m), drp (m): shared workspaces; cp: output (n x m).
__device__ void pdir32(const float2* __restrict__ go, int n, int m, float abs_drop, float2* G, const float2* cx,
                       float2* z, float2* gz, float2* Mm, float2* tmp, float* Dd, int* drp, float2* __restrict__ cp) {
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += SR_THREADS) {  // GO, symmetrised
    const int r = t / n, q = t - (t / n) * n;
    const float2 g1 = go[r * n + q], g2 = go[q * n + r];
    G[r * SR_LD + q] = make_float2(0.5f * (g1.x + g2.x), 0.5f * (g1.y - g2.y));
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += SR_THREADS) {  // M = cX^H GO E
    const int i = t / m, j = t - (t / m) * m;
    float2 s = make_float2(0.f, 0.f);
    for (int r = 0; r < n; ++r) cfmac(s, cx[r * m + i], G[r * SR_LD + j]);
    Mm[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < n * m; t += SR_THREADS) {  // Z = E - cX M
    const int r = t / m, j = t - (t / m) * m;
    float2 s = make_float2(r == j ? 1.f : 0.f, 0.f);
    for (int i = 0; i < m; ++i) {
      const float2 v = cmul(cx[r * m + i], Mm[i * m + j]);
      s.x -= v.x;
      s.y -= v.y;
    }
    z[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < n * m; t += SR_THREADS) {  // GZ = GO Z
    const int r = t / m, j = t - (t / m) * m;
    float2 s = make_float2(0.f, 0.f);
    for (int q = 0; q < n; ++q) cfma(s, G[r * SR_LD + q], z[q * m + j]);
    gz[t] = s;
  }
  __syncthreads();
  for (int i = tid; i < m; i += SR_THREADS) {  // column scales of H = Z^H GZ
    float2 s = make_float2(0.f, 0.f);
    for (int r = 0; r < n; ++r) cfmac(s, z[r * m + i], gz[r * m + i]);
    Dd[i] = (s.x > abs_drop && s.x == s.x) ? 1.f / sqrtf(s.x) : 0.f;
    drp[i] = 0;
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += SR_THREADS) {  // H, unit-diagonal scaled and symmetrised
    const int i = t / m, j = t - (t / m) * m;
    float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
    for (int r = 0; r < n; ++r) {
      cfmac(s1, z[r * m + i], gz[r * m + j]);
      cfmac(s2, z[r * m + j], gz[r * m + i]);
    }
    const float sc = Dd[i] * Dd[j] * 0.5f;
    Mm[t] = make_float2((s1.x + s2.x) * sc, (s1.y - s2.y) * sc);
  }
  __syncthreads();
  chol_drop<float>(Mm, m, m, 1e-10f, drp);
  tri_inv_lower<float>(Mm, m, m, tmp);
  for (int t = tid; t < n * m; t += SR_THREADS) {  // cP = Z T, T[i][c] = D_i conj(Li[c][i]) for c >= i
    const int r = t / m, c = t - (t / m) * m;
    float2 s = make_float2(0.f, 0.f);
    if (!drp[c] && Dd[c] != 0.f) {
      for (int i = 0; i <= c; ++i) {
        const float2 li = Mm[c * m + i];
        cfma(s, z[r * m + i], make_float2(li.x * Dd[i], -li.y * Dd[i]));
      }
    }
    cp[t] = s;
  }
}

}  // namespace

__global__ __launch_bounds__(SR_THREADS) void k_small_rr32(const float2* __restrict__ GA, const float2* __restrict__ GO,
                                                         int n, int m, float drop_tol, const int* __restrict__ kdone,
                                                         float* __restrict__ lam_out, float2* __restrict__ coef,
                                                         float2* __restrict__ cpo, float pdir_abs, int* status,
                                                         double* flops) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* B0 = (float2*)smem;          // GO -> L -> Jacobi buffer 1
  float2* B1 = B0 + SR_MAT;            // GA -> T = L^-1 GA -> Jacobi buffer 0
  float2* Vt = B1 + SR_MAT;            // V^T = conj(L^-1), then rotated (rows: coordinates)
  float2* Cm = Vt + SR_MAT;            // C = L^-1 GA L^-H (original order)
  Plane* pl = (Plane*)(Cm + SR_MAT);   // 2 x 36 planes (by round parity)
  float* D = (float*)(pl + 2 * 36);    // SR_NMAX
  float* ev = D + SR_NMAX;             // SR_NMAX
  int* drop = (int*)(ev + SR_NMAX);    // SR_NMAX
  int* idx = drop + SR_NMAX;           // 2 x SR_NMAX: position -> coordinate (-1: padding)
  int* perm = idx + 2 * SR_NMAX;       // SR_NMAX
  int* npos = perm + SR_NMAX;          // SR_NMAX: position in the next round
  int* ppos = npos + SR_NMAX;          // SR_NMAX: position in the previous round
  int* blk = ppos + SR_NMAX;           // SR_BLK: upper blocks t1 | t2 << 8, row-major
  int* misc = blk + SR_BLK;            // [0] kept count, [2] floor bits
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int k = blockIdx.x;
  const float2* ga = GA + (long long)k * n * n;
  const float2* go = GO + (long long)k * n * n;
  float2* ck = coef + (long long)k * n * m;
  float2* cpk = cpo ? cpo + (long long)k * n * m : nullptr;  // conjugate-direction coefficients (or none)
  if (kdone && kdone[k]) {  // locked k-point: keep its block, leave lambda untouched, no conjugate block
    for (int t = tid; t < n * m; t += blockDim.x) {
      const int i = t / m, j = t % m;
      ck[t] = make_float2(i == j ? 1.f : 0.f, 0.f);
      if (cpk) cpk[t] = make_float2(0.f, 0.f);
    }
    return;
  }
  // 1. scaling, symmetrised copies, identity right-hand side of L^-1 (in Vt)
  for (int i = tid; i < n; i += blockDim.x) {
    const float d = go[i * n + i].x;
    D[i] = (d > 0.f && d == d) ? 1.f / sqrtf(d) : 0.f;
    drop[i] = 0;
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += blockDim.x) {
    const int i = t / n, c = t % n;
    const float2 a1 = ga[i * n + c], a2 = ga[c * n + i];
    const float2 b1 = go[i * n + c], b2 = go[c * n + i];
    const float s = D[i] * D[c] * 0.5f;
    B1[i * SR_LD + c] = make_float2((a1.x + a2.x) * s, (a1.y - a2.y) * s);
    B0[i * SR_LD + c] = make_float2((b1.x + b2.x) * s, (b1.y - b2.y) * s);
    Vt[i * SR_LD + c] = make_float2(i == c ? 1.f : 0.f, 0.f);
  }
  for (int t = tid; t < n * (SR_NMAX - n); t += blockDim.x)  // padding columns n .. 71
    Vt[(t / (SR_NMAX - n)) * SR_LD + n + t % (SR_NMAX - n)] = make_float2(0.f, 0.f);
  __syncthreads();
  // 2. blocked Cholesky of B0 (lower)
  for (int j0 = 0; j0 < n; j0 += SR_PB) {
    const int j1 = min(j0 + SR_PB, n);
    if (warp == 0) {
      for (int j = j0; j < j1; ++j) {
        const float d = B0[j * SR_LD + j].x;
        if (!(d > drop_tol)) {  // dropped: no update; its row and column are reset below
          if (lane == 0) drop[j] = 1;
          __syncwarp();
          continue;
        }
        const float sq = sqrtf(d), inv = 1.f / sq;
        for (int i = j + 1 + lane; i < n; i += 32) {
          const float2 v = B0[i * SR_LD + j];
          B0[i * SR_LD + j] = make_float2(v.x * inv, v.y * inv);
        }
        if (lane == 0) B0[j * SR_LD + j] = make_float2(sq, 0.f);
        __syncwarp();
        for (int c = j + 1; c < j1; ++c) {
          const float2 lc = B0[c * SR_LD + j];
          for (int i = c + lane; i < n; i += 32) {
            const float2 li = B0[i * SR_LD + j];
            float2 v = B0[i * SR_LD + c];
            v.x -= li.x * lc.x + li.y * lc.y;  // v -= li conj(lc)
            v.y -= li.y * lc.x - li.x * lc.y;
            B0[i * SR_LD + c] = v;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // trailing update of rows and columns >= j1 by the panel's kept columns
    const int nt = n - j1;
    for (int r = warp; r < nt; r += 32) {
      const int i = j1 + r;
      for (int q = lane; q <= r; q += 32) {
        const int c = j1 + q;
        float2 v = B0[i * SR_LD + c];
        for (int jj = j0; jj < j1; ++jj) {
          if (drop[jj]) continue;
          const float2 li = B0[i * SR_LD + jj], lc = B0[c * SR_LD + jj];
          v.x -= li.x * lc.x + li.y * lc.y;
          v.y -= li.y * lc.x - li.x * lc.y;
        }
        B0[i * SR_LD + c] = v;
      }
    }
    __syncthreads();
  }
  // dropped coordinates: row and column of L become e_j
  for (int t = tid; t < n * n; t += blockDim.x) {
    const int i = t / n, c = t % n;
    if (c <= i && (drop[i] || drop[c])) B0[i * SR_LD + c] = make_float2(i == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // 3. T = L^-1 GA (in place in B1) and L^-1 (in place in Vt), then C = L^-1 T^H in Cm
  {
    float2* const P[2] = {B1, Vt};
    block_forward(B0, P, n, n, 2 * n);
  }
  for (int t = tid; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t % n;
    Cm[i * SR_LD + j] = zconj(B1[j * SR_LD + i]);
    Vt[i * SR_LD + j] = zconj(Vt[i * SR_LD + j]);  // V^T = conj(L^-1)
  }
  __syncthreads();
  {
    float2* const P[2] = {Cm, Cm};
    block_forward(B0, P, n, n, n);
  }
  if (tid == 0) {
    int kept = 0;
    for (int i = 0; i < n; ++i)
      if (!drop[i]) idx[kept++] = i;
    misc[0] = kept;
    if (kept & 1) idx[kept] = -1;  // padding position
  }
  __syncthreads();
  const int nk_ = misc[0];
  if (nk_ < m) {
    // too few independent directions: keep the current block (identity on its first m coordinates)
    for (int t = tid; t < n * m; t += blockDim.x) {
      const int i = t / m, j = t % m;
      ck[t] = make_float2(i == j ? 1.f : 0.f, 0.f);
    }
    for (int j = tid; j < m; j += blockDim.x) lam_out[(long long)k * m + j] = ga[j * n + j].x / go[j * n + j].x;
    if (tid == 0) set_status(status, PC_ENOCONV);
    if (cpk) {
      for (int t = tid; t < n * m; t += blockDim.x) {
        const int i = t / m, j = t % m;
        B1[t] = make_float2(i == j ? 1.f : 0.f, 0.f);
      }
      __syncthreads();
      pdir32(go, n, m, pdir_abs, B0, B1, B1 + n * m, B1 + 2 * n * m, Cm, Cm + m * m, ev, drop, cpk);
    }
    return;
  }
  const int npad = nk_ + (nk_ & 1), np = npad / 2, nrounds = npad - 1;
  const int nblk = np * (np + 1) / 2;
  // 4. packed position-ordered upper copy in B1 (T is no longer needed) and the round tables
  for (int t = tid; t < npad * npad; t += blockDim.x) {
    const int i = t / npad, j = t % npad;
    if (i <= j) {
      const int a = idx[i], b = idx[j];
      float2 v = (a < 0 || b < 0) ? make_float2(0.f, 0.f) : Cm[a * SR_LD + b];
      if (i == j) v.y = 0.f;
      B1[i * SR_LD + j] = v;
    }
  }
  for (int p = tid; p < npad; p += blockDim.x) {
    npos[p] = next_pos(p, np);
    ppos[p] = prev_pos(p, np);
  }
  for (int t1 = tid; t1 < np; t1 += blockDim.x) {
    const int base = t1 * np - t1 * (t1 - 1) / 2;  // first block of row t1
    for (int t2 = t1; t2 < np; ++t2) blk[base + t2 - t1] = t1 | (t2 << 8);
  }
  __syncthreads();
  // rounding floor: eps * max |a_ii| over the kept coordinates of the current Ritz block
  if (warp == 0) {
    float mx = 0.f;
    for (int p = lane; p < nk_; p += 32)
      if (idx[p] < m) mx = fmaxf(mx, fabsf(B1[p * SR_LD + p].x));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) misc[2] = __float_as_int(1.1920929e-07f * mx);
  }
  __syncthreads();
  const float floor_abs = __int_as_float(misc[2]);
  if (tid < np) {  // planes of the first round
    const int u = 2 * tid, v = u + 1;
    const bool valid = idx[u] >= 0 && idx[v] >= 0;
    pl[tid] = make_plane(B1[u * SR_LD + u].x, B1[v * SR_LD + v].x, B1[u * SR_LD + v], floor_abs, valid);
  }
  __syncthreads();
  // Jacobi sweeps.  Every round, the last pw warps compute the planes of the next round, three
  // lanes per plane (a_uu, a_vv, a_uv of the rotated matrix, combined by shuffles), ten planes per
  // warp; the other threads take the remaining work list: the upper 2 x 2 blocks of the matrix and
  // (plane, six-column group) updates of V^T, units tid, tid + nthr_o, ...  V^T units:
  // v = plane * nq + group, decoded with a multiply-shift (exact for v < 2^11 and nq <= 12: the
  // rounding error of 2^20 / nq times v stays below 1 / nq).
  const int nq = (n + 5) / 6;
  const int pw = (np + 9) / 10;
  const int nthr_o = SR_THREADS - 32 * pw;
  const int nunits = nblk + np * nq;
  const unsigned vinv = (1u << 20) / (unsigned)nq + 1u;
  const bool plane_warp = warp >= SR_THREADS / 32 - pw;
  const int pt = (warp - (SR_THREADS / 32 - pw)) * 10 + lane / 3;  // plane of this lane
  const int pe = lane % 3;                                          // 0: a_uu, 1: a_vv, 2: a_uv
  const int pbase = lane - pe;
  float2* Scur = B1;
  float2* Snxt = B0;
  int par = 0;
  int sweeps = 0;
  for (int sweep = 0; sweep < SR_MAX_SWEEPS; ++sweep) {
    for (int round = 0; round < nrounds; ++round) {
      const Plane* cur = pl + par * 36;
      Plane* nxt = pl + (par ^ 1) * 36;
      const int* icur = idx + par * SR_NMAX;
      int* inxt = idx + (par ^ 1) * SR_NMAX;
      if (plane_warp) {
        // plane pt of the next round: its positions come from u0, v0 of this round
        const bool mine = lane < 30 && pt < np;
        float2 e = make_float2(0.f, 0.f);
        int u0 = 0, v0 = 0;
        if (mine) {
          u0 = ppos[2 * pt];
          v0 = ppos[2 * pt + 1];
          e = pe == 0 ? rotated_entry(Scur, cur, u0, u0)
                      : (pe == 1 ? rotated_entry(Scur, cur, v0, v0) : rotated_entry(Scur, cur, u0, v0));
        }
        const float auu = __shfl_sync(0xffffffffu, e.x, pbase & 31);
        const float avv = __shfl_sync(0xffffffffu, e.x, (pbase + 1) & 31);
        const float2 auv = make_float2(__shfl_sync(0xffffffffu, e.x, (pbase + 2) & 31),
                                       __shfl_sync(0xffffffffu, e.y, (pbase + 2) & 31));
        if (mine && pe == 0) {
          const bool valid = icur[u0] >= 0 && icur[v0] >= 0;
          nxt[pt] = make_plane(auu, avv, auv, floor_abs, valid);
        }
      } else {
        if (tid < npad) inxt[npos[tid]] = icur[tid];
        for (int u = tid; u < nunits; u += nthr_o) {
          if (u < nblk) {
            const int bt = blk[u];
            const int t1 = bt & 255, t2 = bt >> 8;
            const Plane p1 = cur[t1], p2 = cur[t2];
            const int a0 = 2 * t1, b0 = 2 * t2;
            const int ra = npos[a0], rb = npos[a0 + 1];
            const float4 r0 = *reinterpret_cast<const float4*>(Scur + a0 * SR_LD + b0);
            const float4 r1 = *reinterpret_cast<const float4*>(Scur + (a0 + 1) * SR_LD + b0);
            if (t1 == t2) {
              const float2 m00 = make_float2(r0.x, r0.y), m01 = make_float2(r0.z, r0.w);
              const float2 m10 = zconj(m01), m11 = make_float2(r1.z, r1.w);
              const float2 y00 = col_rot(m00, m01, p2, 0), y10 = col_rot(m10, m11, p2, 0);
              const float2 y01 = col_rot(m00, m01, p2, 1), y11 = col_rot(m10, m11, p2, 1);
              const float2 e00 = row_rot(y00, y10, p1, 0), e11 = row_rot(y01, y11, p1, 1);
              const float2 e01 = p1.on ? make_float2(0.f, 0.f) : row_rot(y01, y11, p1, 0);
              Snxt[ra * SR_LD + ra] = make_float2(e00.x, 0.f);
              Snxt[rb * SR_LD + rb] = make_float2(e11.x, 0.f);
              const bool sw = ra > rb;
              Snxt[(sw ? rb : ra) * SR_LD + (sw ? ra : rb)] = sw ? zconj(e01) : e01;
            } else {
              const int ca = npos[b0], cb = npos[b0 + 1];
              const float2 m00 = make_float2(r0.x, r0.y), m01 = make_float2(r0.z, r0.w);
              const float2 m10 = make_float2(r1.x, r1.y), m11 = make_float2(r1.z, r1.w);
              const float2 y00 = col_rot(m00, m01, p2, 0), y10 = col_rot(m10, m11, p2, 0);
              const float2 y01 = col_rot(m00, m01, p2, 1), y11 = col_rot(m10, m11, p2, 1);
              const float2 e00 = row_rot(y00, y10, p1, 0), e01 = row_rot(y01, y11, p1, 0);
              const float2 e10 = row_rot(y00, y10, p1, 1), e11 = row_rot(y01, y11, p1, 1);
              bool sw;
              sw = ra > ca; Snxt[(sw ? ca : ra) * SR_LD + (sw ? ra : ca)] = sw ? zconj(e00) : e00;
              sw = ra > cb; Snxt[(sw ? cb : ra) * SR_LD + (sw ? ra : cb)] = sw ? zconj(e01) : e01;
              sw = rb > ca; Snxt[(sw ? ca : rb) * SR_LD + (sw ? rb : ca)] = sw ? zconj(e10) : e10;
              sw = rb > cb; Snxt[(sw ? cb : rb) * SR_LD + (sw ? rb : cb)] = sw ? zconj(e11) : e11;
            }
          } else {
            const unsigned v = (unsigned)(u - nblk);
            const int t = (int)((v * vinv) >> 20);
            const int h = (int)v - t * nq;
            const Plane w = cur[t];
            if (w.on) {
              // rows p, q of V^T, elements 6h .. 6h + 5 (columns n .. 71 are zero padding)
              float4* vp4 = reinterpret_cast<float4*>(Vt + icur[2 * t] * SR_LD + 6 * h);
              float4* vq4 = reinterpret_cast<float4*>(Vt + icur[2 * t + 1] * SR_LD + 6 * h);
              const float2 sc = zconj(w.s);
#pragma unroll
              for (int g = 0; g < 3; ++g) {
                const float4 a = vp4[g], b = vq4[g];
                const float2 p0 = zaxpy(w.c, make_float2(a.x, a.y), zneg(zmul(sc, make_float2(b.x, b.y))));
                const float2 p1_ = zaxpy(w.c, make_float2(a.z, a.w), zneg(zmul(sc, make_float2(b.z, b.w))));
                const float2 q0 = zaxpy(w.c, make_float2(b.x, b.y), zmul(w.s, make_float2(a.x, a.y)));
                const float2 q1 = zaxpy(w.c, make_float2(b.z, b.w), zmul(w.s, make_float2(a.z, a.w)));
                vp4[g] = make_float4(p0.x, p0.y, p1_.x, p1_.y);
                vq4[g] = make_float4(q0.x, q0.y, q1.x, q1.y);
              }
            }
          }
        }
      }
      __syncthreads();
      float2* t_ = Scur; Scur = Snxt; Snxt = t_;
      par ^= 1;
    }
    sweeps = sweep + 1;
    // converged when no pair of the current matrix would rotate
    bool any = false;
    const int* icur = idx + par * SR_NMAX;
    for (int t = tid; t < npad * npad; t += blockDim.x) {
      const int i = t / npad, j = t % npad;
      if (i < j && icur[i] >= 0 && icur[j] >= 0) {
        const float2 a = Scur[i * SR_LD + j];
        const float beta = sqrtf(a.x * a.x + a.y * a.y);
        any |= beta > 1.1920929e-07f * sqrtf(fabsf(Scur[i * SR_LD + i].x) * fabsf(Scur[j * SR_LD + j].x)) + floor_abs;
      }
    }
    if (!__syncthreads_or(any)) break;
  }
  // 5. lowest m eigenpairs of the kept coordinates
  const int* icur = idx + par * SR_NMAX;
  for (int p = tid; p < npad; p += blockDim.x) ev[p] = Scur[p * SR_LD + p].x;
  __syncthreads();
  for (int p = tid; p < npad; p += blockDim.x) {
    if (icur[p] < 0) continue;
    int r = 0;
    const float vi = ev[p];
    for (int q = 0; q < npad; ++q) {
      if (icur[q] < 0) continue;
      r += (ev[q] < vi || (ev[q] == vi && icur[q] < icur[p])) ? 1 : 0;
    }
    perm[r] = p;
  }
  __syncthreads();
  for (int t = tid; t < n * m; t += blockDim.x) {
    const int i = t / m, j = t % m;
    const float2 v = Vt[icur[perm[j]] * SR_LD + i];  // V[i][col] = V^T[col][i]
    const float2 c = make_float2(v.x * D[i], v.y * D[i]);
    ck[t] = c;
    B1[t] = c;  // the Jacobi buffers are free: cX for the conjugate directions
  }
  for (int j = tid; j < m; j += blockDim.x) lam_out[(long long)k * m + j] = ev[perm[j]];
  if (cpk) {
    __syncthreads();
    pdir32(go, n, m, pdir_abs, B0, B1, B1 + n * m, B1 + 2 * n * m, Cm, Cm + m * m, ev, drop, cpk);
  }
  if (flops && tid == 0) {
    // algorithmic work: Cholesky n^3/6, L^-1 GA n^3/2, L^-1 T^H n^3/2 and L^-1 n^3/6 complex
    // multiply-adds (8 real flops each); per Jacobi sweep n_k (n_k - 1) / 2 rotations, each
    // updating 2 n_k entries of C and 2 n entries of V at 12 real flops per entry
    const double nn = n, kk = nk_;
    atomicAdd(flops, 8.0 * (4.0 / 3.0) * nn * nn * nn + sweeps * kk * (kk - 1.0) * 0.5 * 24.0 * (kk + nn));
  }
}

int launch_small_rr32(const float2* GA, const float2* GO, int n, int m, int nk, float drop_tol, const int* kdone,
                      float* lam_out, float2* coef, float2* cp, float pdir_abs, int* status, double* flops,
                      cudaStream_t s) {
  if (n > SR_NMAX || m > n || n < 1) return PC_EINVAL;
  const size_t sm = sizeof(float2) * 4 * (size_t)SR_MAT + sizeof(Plane) * 72 + sizeof(float) * 2 * SR_NMAX +
                    sizeof(int) * (7 * SR_NMAX + SR_BLK + 8);
  static const cudaError_t attr =  // once, thread-safe (k groups launch from several host threads)
      cudaFuncSetAttribute(k_small_rr32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  (void)attr;
  k_small_rr32<<<nk, SR_THREADS, sm, s>>>(GA, GO, n, m, drop_tol, kdone, lam_out, coef, cp, pdir_abs, status, flops);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
