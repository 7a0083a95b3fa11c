// Small dense Hermitian algebra in shared memory for one CTA (any block size): Cholesky with
// column dropping and the in-place inverse of a lower-triangular factor.  Shared by the
// projected-problem kernels of both precisions.
#pragma once
#include "kernels.h"

// Cholesky of Hermitian B (n x n, stride ld) with column dropping, in place (lower
// triangle); drop[j] = 1 for a pivot at or below tol (dropped rows/columns become e_j).
template <typename R>
__device__ void chol_drop(typename cplx_t<R>::type* B, int n, int ld, R tol, int* drop) {
  typedef typename cplx_t<R>::type C2;
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    R d = B[j * ld + j].x;
    bool dr = !(d > tol);
    __syncthreads();
    if (dr) {
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (i != j) { B[i * ld + j] = mk<R>(0, 0); B[j * ld + i] = mk<R>(0, 0); }
      if (threadIdx.x == 0) { B[j * ld + j] = mk<R>(1, 0); drop[j] = 1; }
      continue;
    }
    R sq = sqrt(d), inv = (R)1 / sq;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) B[i * ld + j] = cscale(B[i * ld + j], inv);
    if (threadIdx.x == 0) B[j * ld + j] = mk<R>(sq, 0);
    __syncthreads();
    int nt = n - j - 1;
    for (int t = threadIdx.x; t < nt * nt; t += blockDim.x) {
      int i = j + 1 + t / nt, c = j + 1 + t % nt;
      if (c <= i) {
        C2 v = B[i * ld + c];
        C2 l1 = B[i * ld + j], l2 = B[c * ld + j];
        v.x -= l1.x * l2.x + l1.y * l2.y;
        v.y -= l1.y * l2.x - l1.x * l2.y;
        B[i * ld + c] = v;
      }
    }
  }
  __syncthreads();
}

// In-place inverse of the lower-triangular L (n x n, stride ld); upper triangle zeroed.
// Column j of the inverse from columns j+1.. (already inverted): one warp per row, lanes
// split the dot product and reduce with shuffles.
template <typename R>
__device__ void tri_inv_lower(typename cplx_t<R>::type* L, int n, int ld, typename cplx_t<R>::type* tmp) {
  typedef typename cplx_t<R>::type C2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = n - 1; j >= 0; --j) {
    __syncthreads();
    C2 ljj = L[j * ld + j];
    R den = ljj.x * ljj.x + ljj.y * ljj.y;
    C2 ajj = mk<R>(ljj.x / den, -ljj.y / den);
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) tmp[i] = L[i * ld + j];
    __syncthreads();
    // new L[i][j] = -ajj * sum_{c=j+1..i} Linv[i][c] * old L[c][j]
    for (int i = j + 1 + warp; i < n; i += nw) {
      C2 s = mk<R>(0, 0);
      for (int c = j + 1 + lane; c <= i; c += 32) cfma(s, L[i * ld + c], tmp[c]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) {
        C2 v = cmul(s, ajj);
        L[i * ld + j] = mk<R>(-v.x, -v.y);
      }
    }
    if (threadIdx.x == 0) L[j * ld + j] = ajj;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, c = t % n;
    if (c > i) L[i * ld + c] = mk<R>(0, 0);
  }
  __syncthreads();
}
