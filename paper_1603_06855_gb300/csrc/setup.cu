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
// SIMP interpolation: fields[0] = density, fields[1] = f1, fields[2] = f2 per element.
__global__ void k_interp(const double* __restrict__ rho, int ne, MaterialConsts mc,
                         double* __restrict__ fields, double* __restrict__ dchi,
                         double* __restrict__ chi_out, int* status) {
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
  fields[ne + e] = mc.f1_0 + chi * (mc.f1_1 - mc.f1_0);
  fields[2 * ne + e] = mc.f2_0 + chi * (mc.f2_1 - mc.f2_0);
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

// In-place Gauss-Jordan inversion of Hermitian positive definite matrices (no pivoting
// is needed for HPD).  Step k turns column k into the inverse's column k.  The pivot
// row and column are read from a snapshot written by the previous step, so one launch
// per pivot suffices; blockIdx.z selects the matrix.
__global__ void k_gj_snapshot(const double2* __restrict__ A, int N, long long mstride,
                              double2* __restrict__ rowbuf, double2* __restrict__ colbuf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int z = blockIdx.z;
  if (i >= N) return;
  rowbuf[(long long)z * N + i] = A[z * mstride + i];                 // row 0
  colbuf[(long long)z * N + i] = A[z * mstride + (long long)i * N];  // column 0
}

__global__ void k_gj_step(double2* __restrict__ A, int N, long long mstride, int k,
                          const double2* __restrict__ row_in, const double2* __restrict__ col_in,
                          double2* __restrict__ row_out, double2* __restrict__ col_out) {
  __shared__ double2 ip_s;
  const int z = blockIdx.z;
  const double2* rk = row_in + (long long)z * N;
  const double2* ck = col_in + (long long)z * N;
  if (threadIdx.x == 0) {  // 1 / pivot, once per block (FP64 division is expensive here)
    double2 piv = rk[k];
    double den = piv.x * piv.x + piv.y * piv.y;
    ip_s = make_double2(piv.x / den, -piv.y / den);
  }
  __syncthreads();
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= N) return;
  const double2 ip = ip_s;
  double2* a = A + z * mstride + (long long)i * N + j;
  double2 v;
  if (i == k && j == k) v = ip;
  else if (i == k) v = cmul(rk[j], ip);
  else if (j == k) v = cmul(make_double2(-ck[i].x, -ck[i].y), ip);
  else v = csub(*a, cmul(ck[i], cmul(rk[j], ip)));
  *a = v;
  if (k + 1 < N) {
    if (i == k + 1) row_out[(long long)z * N + j] = v;
    if (j == k + 1) col_out[(long long)z * N + i] = v;
  }
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
  k_interp<<<cdiv(ne, 256), 256, 0, s>>>(a.rho, ne, a.mc, a.fields, a.dchi, a.chi, a.status);
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
  dim3 gs(cdiv(N, 256), 1, 2);
  k_gj_snapshot<<<gs, 256, 0, s>>>(a.W, N, NN, a.gj_row, a.gj_col);
  PC_LAUNCH_CHECK();
  for (int k = 0; k < N; ++k) {
    dim3 g(cdiv(N, 256), N, 2);
    const double2* rin = a.gj_row + (k & 1) * 2LL * N;
    const double2* cin = a.gj_col + (k & 1) * 2LL * N;
    double2* rout = a.gj_row + ((k + 1) & 1) * 2LL * N;
    double2* cout = a.gj_col + ((k + 1) & 1) * 2LL * N;
    k_gj_step<<<g, 256, 0, s>>>(a.W, N, NN, k, rin, cin, rout, cout);
  }
  PC_LAUNCH_CHECK();
  return PC_OK;
}
