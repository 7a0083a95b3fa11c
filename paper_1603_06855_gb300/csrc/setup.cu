// Per-design operator assembly (k-independent):
//   SIMP interpolation           -- Methods, eq. combinematerial (linear in chi = rho^p)
//   structure factors            -- Methods, eq. loop: centroid sums of the fields times
//                                   exp(i 2 pi Delta.s_e) for every plane-wave difference Delta
//   Toeplitz operators           -- Results, eqs. intOmega / intPhi via eq. matrixofintegral:
//                                   T_c[p][q] = V c^(g_q - g_p)
//   inverse compliance operators -- the stress elimination of eq. matrixform; both phases are
//                                   isotropic, so Phi^-1 only needs the inverses of the bulk
//                                   (f1 = (1-2nu)/E) and shear (f2 = (1+nu)/E) Toeplitz blocks.
#include "kernels.h"

// ---------------------------------------------------------------------------
// SIMP interpolation: fields[0] = density, fields[1] = f1, fields[2] = f2 per element, and
// dfc = (d f1 / d chi, d f2 / d chi) per element (dfc may be NULL).  PC_LAW_COMPLIANCE: f1, f2
// linear in chi; PC_LAW_YOUNG: E and nu linear in chi, f1 = (1 - 2 nu)/E, f2 = (1 + nu)/E, so
// d f1/d chi = (-2 dnu E - (1 - 2 nu) dE) / E^2 and d f2/d chi = (dnu E - (1 + nu) dE) / E^2.
__global__ void k_interp(const double* __restrict__ rho, int ne, MaterialConsts mc,
                         double* __restrict__ fields, double* __restrict__ dchi,
                         double* __restrict__ chi_out, int* status, double* __restrict__ dfc) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double r = rho[e];
  if (!(r >= 0.0 && r <= 1.0)) {  // also catches NaN
    set_status(status, PC_EDOMAIN);
    r = (r > 1.0) ? 1.0 : 0.0;
    if (!(rho[e] == rho[e])) r = 0.0;
  }
  double chi, dc;
  if (mc.penal == 1.0) { chi = r; dc = 1.0; }
  else { chi = pow(r, mc.penal); dc = (r > 0.0) ? mc.penal * pow(r, mc.penal - 1.0) : 0.0; }
  fields[e] = mc.rho0 + chi * (mc.rho1 - mc.rho0);
  double f1, f2, d1, d2;
  if (mc.law == PC_LAW_YOUNG) {
    const double dE = mc.E1 - mc.E0, dn = mc.nu1 - mc.nu0;
    const double E = mc.E0 + chi * dE, nu = mc.nu0 + chi * dn;
    f1 = (1.0 - 2.0 * nu) / E;
    f2 = (1.0 + nu) / E;
    d1 = (-2.0 * dn * E - (1.0 - 2.0 * nu) * dE) / (E * E);
    d2 = (dn * E - (1.0 + nu) * dE) / (E * E);
  } else {
    f1 = mc.f1_0 + chi * (mc.f1_1 - mc.f1_0);
    f2 = mc.f2_0 + chi * (mc.f2_1 - mc.f2_0);
    d1 = mc.f1_1 - mc.f1_0;
    d2 = mc.f2_1 - mc.f2_0;
  }
  fields[ne + e] = f1;
  fields[2 * ne + e] = f2;
  if (dfc) {
    dfc[e] = d1;
    dfc[ne + e] = d2;
  }
  dchi[e] = dc;
  chi_out[e] = chi;
}

// Mean of chi (deterministic single-block reduction) for the preconditioner's reference medium.
__global__ void k_mean(const double* __restrict__ x, int n, double* out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (double)n;
}

// Structure factors by three separable sums, one grid axis at a time.
// Stage 1 (axis 2): t1[f][i][j][d3] = sum_l c_f[i][j][l] exp(i pi D3 (2l+1)/n2), D3 = d3 - 2M.
__global__ void k_sfac1(const double* __restrict__ fields, int n0, int n1, int n2, int M,
                        double2* __restrict__ t1) {
  int L = 4 * M + 1;
  long long total = 3LL * n0 * n1 * L;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int d3 = (int)(t % L);
  long long r = t / L;           // (f, i, j)
  int D = d3 - 2 * M;
  const double* src = fields + r * n2;
  double2 acc = make_double2(0.0, 0.0);
  for (int l = 0; l < n2; ++l) {
    double2 ph = phase_pi_over((long long)D * (2 * l + 1), n2);
    acc.x = fma(src[l], ph.x, acc.x);
    acc.y = fma(src[l], ph.y, acc.y);
  }
  t1[t] = acc;
}
// Stage 2 (axis 1): t2[f][i][d2][d3] = sum_j t1[f][i][j][d3] exp(i pi D2 (2j+1)/n1).
__global__ void k_sfac2(const double2* __restrict__ t1, int n0, int n1, int M, double2* __restrict__ t2) {
  int L = 4 * M + 1;
  long long total = 3LL * n0 * L * L;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int d3 = (int)(t % L);
  int d2 = (int)((t / L) % L);
  long long fi = t / ((long long)L * L);
  int D = d2 - 2 * M;
  double2 acc = make_double2(0.0, 0.0);
  for (int j = 0; j < n1; ++j) {
    double2 ph = phase_pi_over((long long)D * (2 * j + 1), n1);
    cfma(acc, t1[(fi * n1 + j) * L + d3], ph);
  }
  t2[t] = acc;
}
// Stage 3 (axis 0): sfac[f][d1][d2][d3] = (1/ne) sum_i t2[f][i][d2][d3] exp(i pi D1 (2i+1)/n0).
__global__ void k_sfac3(const double2* __restrict__ t2, int n0, int M, double inv_ne, double2* __restrict__ sf) {
  int L = 4 * M + 1;
  long long L2 = (long long)L * L;
  long long total = 3LL * L * L2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  long long d23 = t % L2;
  int d1 = (int)((t / L2) % L);
  int f = (int)(t / (L2 * L));
  int D = d1 - 2 * M;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = 0; i < n0; ++i) {
    double2 ph = phase_pi_over((long long)D * (2 * i + 1), n0);
    cfma(acc, t2[((long long)f * n0 + i) * L2 + d23], ph);
  }
  sf[t] = cscale(acc, inv_ne);
}

// Toeplitz operators T_f[p][q] = V * c^_f(g_q - g_p), f in {density, f1, f2}, SI units.
__global__ void k_toeplitz(const double2* __restrict__ sf, int M, double V, double2* __restrict__ T) {
  int M2 = 2 * M + 1, N = M2 * M2 * M2, L = 4 * M + 1;
  long long NN = (long long)N * N;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * NN) return;
  int f = (int)(t / NN);
  long long pq = t % NN;
  int p = (int)(pq / N), q = (int)(pq % N);
  int p1 = p / (M2 * M2), p2 = (p / M2) % M2, p3 = p % M2;
  int q1 = q / (M2 * M2), q2 = (q / M2) % M2, q3 = q % M2;
  int d1 = q1 - p1 + 2 * M, d2 = q2 - p2 + 2 * M, d3 = q3 - p3 + 2 * M;
  double2 v = sf[(long long)f * L * L * L + ((long long)d1 * L + d2) * L + d3];
  T[t] = cscale(v, V);
}

// In-place blocked Gauss-Jordan inversion of Hermitian positive definite matrices (no
// pivoting is needed for HPD).  For the pivot block [k0, k0 + bb) with P = A11^-1, one panel
// step maps
//   A11 <- P,   A1j <- P A1j,   Ai1 <- -Ai1 P,   Aij <- Aij - Ai1 P A1j   (i, j outside the block),
// which is bb scalar Gauss-Jordan steps at once.  Three launches per panel: the pivot block
// inverse (with a copy of the old pivot rows), the column panel Ai1 P, and the update of the
// whole matrix.  blockIdx.z selects the matrix.
#define GJ_B 32
__global__ void k_gj_pivot(const double2* __restrict__ A, int N, long long mstride, int k0, int bb,
                           double2* __restrict__ Pbuf, double2* __restrict__ Ar) {
  __shared__ double2 P[GJ_B * (GJ_B + 1)];
  __shared__ double2 prow[GJ_B], pcol[GJ_B], qrow[GJ_B];
  __shared__ double2 sip;
  const int z = blockIdx.z;
  const double2* Az = A + z * mstride;
  const int ld = GJ_B + 1;
  for (int t = threadIdx.x; t < bb * bb; t += blockDim.x) {
    int r = t / bb, c = t % bb;
    P[r * ld + c] = Az[(long long)(k0 + r) * N + k0 + c];
  }
  // old pivot rows for the update of the rest of the matrix
  double2* arz = Ar + (long long)z * GJ_B * N;
  for (long long t = threadIdx.x; t < (long long)bb * N; t += blockDim.x) {
    int r = (int)(t / N), c = (int)(t % N);
    arz[(long long)r * N + c] = Az[(long long)(k0 + r) * N + c];
  }
  __syncthreads();
  // One scalar step per pivot k.  The reciprocal of the pivot and the scaled pivot row
  // q_c = prow_c / piv are formed once (FP64 division and complex products are scarce on one SM's
  // FP64 pipe), then every element takes its update.
  for (int k = 0; k < bb; ++k) {
    if ((int)threadIdx.x < bb) {
      prow[threadIdx.x] = P[k * ld + threadIdx.x];
      pcol[threadIdx.x] = P[threadIdx.x * ld + k];
    }
    if (threadIdx.x == 0) {
      const double2 piv = P[k * ld + k];
      const double den = piv.x * piv.x + piv.y * piv.y;
      sip = make_double2(piv.x / den, -piv.y / den);
    }
    __syncthreads();
    const double2 ip = sip;
    if ((int)threadIdx.x < bb) qrow[threadIdx.x] = cmul(prow[threadIdx.x], ip);
    __syncthreads();
    for (int t = threadIdx.x; t < bb * bb; t += blockDim.x) {
      int r = t / bb, c = t % bb;
      double2 v;
      if (r == k && c == k) v = ip;
      else if (r == k) v = qrow[c];
      else if (c == k) v = cmul(make_double2(-pcol[r].x, -pcol[r].y), ip);
      else v = csub(P[r * ld + c], cmul(pcol[r], qrow[c]));
      P[r * ld + c] = v;
    }
    __syncthreads();
  }
  double2* pz = Pbuf + (long long)z * GJ_B * GJ_B;
  for (int t = threadIdx.x; t < bb * bb; t += blockDim.x) pz[t] = P[(t / bb) * ld + t % bb];
}

// Cp[i][l] = sum_m A[i][k0 + m] P[m][l]: the old column panel times the pivot-block inverse.
__global__ void k_gj_colpanel(const double2* __restrict__ A, int N, long long mstride, int k0, int bb,
                              const double2* __restrict__ Pbuf, double2* __restrict__ Cp) {
  const int z = blockIdx.z;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * bb) return;
  const int i = (int)(t / bb), l = (int)(t % bb);
  const double2* arow = A + z * mstride + (long long)i * N + k0;
  const double2* pz = Pbuf + (long long)z * GJ_B * GJ_B;
  double2 acc = make_double2(0.0, 0.0);
  for (int m = 0; m < bb; ++m) cfma(acc, arow[m], pz[m * bb + l]);
  Cp[(long long)z * GJ_B * N + (long long)i * GJ_B + l] = acc;
}

// Update of one panel step for a set of rows, one row per blockIdx.y: rows r0 + y, except that
// the nskip rows from skip0 on are stepped over (y >= skip0 - r0 maps to y + nskip).
__global__ void k_gj_update(double2* __restrict__ A, int N, long long mstride, int k0, int bb,
                            const double2* __restrict__ Pbuf, const double2* __restrict__ Ar,
                            const double2* __restrict__ Cp, int r0, int skip0, int nskip) {
  __shared__ double2 crow[GJ_B];
  const int z = blockIdx.z;
  int i = r0 + (int)blockIdx.y;
  if (i >= skip0) i += nskip;
  const double2* arz = Ar + (long long)z * GJ_B * N;
  const double2* pz = Pbuf + (long long)z * GJ_B * GJ_B;
  const bool iblk = i >= k0 && i < k0 + bb;
  if ((int)threadIdx.x < bb)
    crow[threadIdx.x] = iblk ? pz[(i - k0) * bb + threadIdx.x] : Cp[(long long)z * GJ_B * N + (long long)i * GJ_B + threadIdx.x];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double2* a = A + z * mstride + (long long)i * N + j;
  const bool jblk = j >= k0 && j < k0 + bb;
  double2 v;
  if (iblk && jblk) {
    v = crow[j - k0];                        // P
  } else if (jblk) {
    const double2 c = crow[j - k0];          // -Ai1 P
    v = make_double2(-c.x, -c.y);
  } else {
    double2 acc = make_double2(0.0, 0.0);    // (P or Ai1 P) times the old pivot rows
    for (int l = 0; l < bb; ++l) cfma(acc, crow[l], arz[(long long)l * N + j]);
    v = iblk ? acc : csub(*a, acc);
  }
  *a = v;
}

// Copies the f1 and f2 Toeplitz operators into the workspace that is inverted in place.
__global__ void k_copy2(const double2* __restrict__ src, double2* __restrict__ dst, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = src[t];
}

// ---------------------------------------------------------------------------
int launch_setup(const SetupArgs& a, cudaStream_t s) {
  const int ne = a.n0 * a.n1 * a.n2;
  const int L = 4 * a.M + 1;
  const int N = (2 * a.M + 1) * (2 * a.M + 1) * (2 * a.M + 1);
  k_interp<<<cdiv(ne, 256), 256, 0, s>>>(a.rho, ne, a.mc, a.fields, a.dchi, a.chi, a.status, a.dfc);
  PC_LAUNCH_CHECK();
  k_mean<<<1, 1024, 0, s>>>(a.chi, ne, a.chi_mean);
  PC_LAUNCH_CHECK();
  long long t1n = 3LL * a.n0 * a.n1 * L;
  k_sfac1<<<cdiv(t1n, 256), 256, 0, s>>>(a.fields, a.n0, a.n1, a.n2, a.M, a.t1);
  PC_LAUNCH_CHECK();
  long long t2n = 3LL * a.n0 * L * L;
  k_sfac2<<<cdiv(t2n, 256), 256, 0, s>>>(a.t1, a.n0, a.n1, a.M, a.t2);
  PC_LAUNCH_CHECK();
  long long sfn = 3LL * L * L * L;
  k_sfac3<<<cdiv(sfn, 256), 256, 0, s>>>(a.t2, a.n0, a.M, 1.0 / (double)ne, a.sfac);
  PC_LAUNCH_CHECK();
  long long NN = (long long)N * N;
  k_toeplitz<<<cdiv(3 * NN, 256), 256, 0, s>>>(a.sfac, a.M, a.V, a.T);
  PC_LAUNCH_CHECK();
  // W1 = T_f1^-1, W2 = T_f2^-1
  k_copy2<<<cdiv(2 * NN, 256), 256, 0, s>>>(a.T + NN, a.W, 2 * NN);
  PC_LAUNCH_CHECK();
  // Scratch of two panels (parity p): pivot-block inverses, column panels, old pivot rows.
  const long long colsz = 2LL * GJ_B * (N + GJ_B), rowsz = 2LL * GJ_B * N;
  double2* Pbuf[2] = {a.gj_col, a.gj_col + colsz};                                   // 2 x GJ_B x GJ_B each
  double2* Cp[2] = {a.gj_col + 2LL * GJ_B * GJ_B, a.gj_col + colsz + 2LL * GJ_B * GJ_B};  // 2 x N x GJ_B
  double2* Ar[2] = {a.gj_row, a.gj_row + rowsz};                                     // 2 x GJ_B x N
  // Look-ahead: the pivot block of panel k + 1 needs only panel k's update of its own rows, so
  // those rows are updated first and the next pivot block (one CTA per matrix) runs on the side
  // stream while the main stream updates the other rows.
  const bool ahead = a.side && a.ev_rows && a.ev_pivot;
  k_gj_pivot<<<dim3(1, 1, 2), 512, 0, s>>>(a.W, N, NN, 0, min(GJ_B, N), Pbuf[0], Ar[0]);
  for (int k0 = 0, pi = 0; k0 < N; k0 += GJ_B, ++pi) {
    const int bb = min(GJ_B, N - k0), p = pi & 1;
    const int kn = k0 + bb, bbn = min(GJ_B, N - kn);
    k_gj_colpanel<<<dim3(cdiv((long long)N * bb, 256), 1, 2), 256, 0, s>>>(a.W, N, NN, k0, bb, Pbuf[p], Cp[p]);
    const dim3 gx(cdiv(N, 256), 1, 2);
    if (bbn > 0 && ahead) {
      k_gj_update<<<dim3(gx.x, bbn, 2), 256, 0, s>>>(a.W, N, NN, k0, bb, Pbuf[p], Ar[p], Cp[p], kn, N, 0);
      PC_CUDA_TRY(cudaEventRecord(a.ev_rows, s));
      PC_CUDA_TRY(cudaStreamWaitEvent(a.side, a.ev_rows, 0));
      k_gj_pivot<<<dim3(1, 1, 2), 512, 0, a.side>>>(a.W, N, NN, kn, bbn, Pbuf[p ^ 1], Ar[p ^ 1]);
      PC_CUDA_TRY(cudaEventRecord(a.ev_pivot, a.side));
      k_gj_update<<<dim3(gx.x, N - bbn, 2), 256, 0, s>>>(a.W, N, NN, k0, bb, Pbuf[p], Ar[p], Cp[p], 0, kn, bbn);
      PC_CUDA_TRY(cudaStreamWaitEvent(s, a.ev_pivot, 0));
    } else {
      k_gj_update<<<dim3(gx.x, N, 2), 256, 0, s>>>(a.W, N, NN, k0, bb, Pbuf[p], Ar[p], Cp[p], 0, N, 0);
      if (bbn > 0) k_gj_pivot<<<dim3(1, 1, 2), 512, 0, s>>>(a.W, N, NN, kn, bbn, Pbuf[p ^ 1], Ar[p ^ 1]);
    }
  }
  PC_LAUNCH_CHECK();
  return PC_OK;
}
