// Gap objective (Methods, eq. obj; omega form of the Results' note on normalized gaps)
// and the adjoint design sensitivities (Methods, eqs. normalev, sensitivityew, diffOmega,
// diffPhi).  With theta^H Omega theta = 1 and s = Phi^-1 H^H theta,
//   d lambda / d rho_e = chi'_e v_e [ -lambda (rho1 - rho0) sum_c |u_c(x_e)|^2
//                                      - f1'_e |sigma_bulk(x_e)|^2 - f2'_e |sigma_dev(x_e)|^2 ],
// f1'_e, f2'_e the derivatives of the compliance moduli with respect to chi at element e (the
// phase differences under the compliance law, per element under eq. combinematerial's law),
// where u and sigma are the displacement and stress fields synthesised at the element
// centroid from the plane-wave coefficients.  The kernels synthesise the 3 + 6 fields of
// every weighted (k, band) on the voxel grid by separable sums (axis 2, axis 1 into a
// scratch array, then axis 0 inside the per-voxel reduction) and reduce the weighted
// quadratic forms over all (k, band): per chunk of pairs, then over the chunks in FP64.
#include <algorithm>
#include "kernels.h"

// ---------------------------------------------------------------------------
__global__ void k_omega(const double* __restrict__ lam_m, int nk, int nb, int m, double lref,
                        double* __restrict__ omega, double* __restrict__ lam_phys, double* __restrict__ lam_nd) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nk * nb) return;
  int k = t / nb, b = t % nb;
  double l = lam_m[k * m + b];
  if (lam_nd) lam_nd[t] = l;
  if (lam_phys) lam_phys[t] = l * lref;
  if (omega) omega[t] = sqrt(fmax(l * lref, 0.0));
}
int launch_omega(const double* lam_m, int nk, int nb, int m, double lref, double* omega, double* lam_nd,
                 cudaStream_t s) {
  k_omega<<<cdiv((long long)nk * nb, 256), 256, 0, s>>>(lam_m, nk, nb, m, lref, omega, nullptr, lam_nd);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// ---------------------------------------------------------------------------
// Gap, weights dG/dlambda (physical) and the compacted list of weighted (k, band).
__global__ void k_gap(GapArgs a) {
  __shared__ double sv[256];
  __shared__ int si[256];
  __shared__ int ka_s, kb_s;
  const int nk = a.nk, nb = a.nb;
  for (int t = threadIdx.x; t < nk * nb; t += blockDim.x) a.weights[t] = 0.0;
  __syncthreads();
  if (a.mode == PC_GRAD_ALLBANDS) {
    double s = 0.0;
    for (int t = threadIdx.x; t < nk * nb; t += blockDim.x) {
      a.weights[t] = a.w_user[t];
      s += a.w_user[t] * a.lam[t] * a.lref;
    }
    sv[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sv[threadIdx.x] += sv[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      *a.gap_out = sv[0];
      int c = 0;
      for (int t = 0; t < nk * nb; ++t)
        if (a.weights[t] != 0.0) a.pairs[c++] = t;
      *a.npairs = c;
    }
    return;
  }
  const int lo = a.n_lower - 1, hi = a.n_lower;
  if (a.mode == PC_GAP_KS_INTERNAL) {
    // Smooth surrogate: with x = omega / omega_ref = sqrt(lam_nd), a = (1/beta) log sum_k
    // exp(beta x_{k,lo}) and b = -(1/beta) log sum_k exp(-beta x_{k,hi}), G = 2 (b - a) / (b + a).
    __shared__ double xm_s, ym_s, sa_s, sb_s;
    const double beta = a.ks_beta;
    double mx = -1e300, my = 1e300;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
      mx = fmax(mx, sqrt(fmax(a.lam[k * nb + lo], 0.0)));
      my = fmin(my, sqrt(fmax(a.lam[k * nb + hi], 0.0)));
    }
    sv[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sv[threadIdx.x] = fmax(sv[threadIdx.x], sv[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) xm_s = sv[0];
    __syncthreads();
    sv[threadIdx.x] = my;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sv[threadIdx.x] = fmin(sv[threadIdx.x], sv[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) ym_s = sv[0];
    __syncthreads();
    const double xm = xm_s, ym = ym_s;
    double pa = 0.0, pb = 0.0;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
      pa += exp(beta * (sqrt(fmax(a.lam[k * nb + lo], 0.0)) - xm));
      pb += exp(-beta * (sqrt(fmax(a.lam[k * nb + hi], 0.0)) - ym));
    }
    sv[threadIdx.x] = pa;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sv[threadIdx.x] += sv[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sa_s = sv[0];
    __syncthreads();
    sv[threadIdx.x] = pb;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sv[threadIdx.x] += sv[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) sb_s = sv[0];
    __syncthreads();
    const double A_ = xm + log(sa_s) / beta, B_ = ym - log(sb_s) / beta;
    const double dGa = -4.0 * B_ / ((A_ + B_) * (A_ + B_)), dGb = 4.0 * A_ / ((A_ + B_) * (A_ + B_));
    if (threadIdx.x == 0) *a.gap_out = 2.0 * (B_ - A_) / (B_ + A_);
    // weights dG/dlambda_phys: p_k dGa / (2 x lref) on band lo, q_k dGb / (2 y lref) on band hi,
    // each shared by the bands of its cluster at that k (one thread per k: no write conflicts)
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
      for (int side = 0; side < 2; ++side) {
        const int band = side == 0 ? lo : hi;
        const double xv = sqrt(fmax(a.lam[k * nb + band], 0.0));
        if (xv <= 0.0) continue;
        const double pw = side == 0 ? exp(beta * (xv - xm)) / sa_s : exp(-beta * (xv - ym)) / sb_s;
        const double wl = (side == 0 ? dGa : dGb) * pw / (2.0 * xv * a.lref);
        const double ref = a.lam[k * nb + band];
        int members = 0;
        for (int b = 0; b < nb; ++b) members += (fabs(a.lam[k * nb + b] - ref) <= a.rel_tol * fabs(ref)) ? 1 : 0;
        for (int b = 0; b < nb; ++b)
          if (fabs(a.lam[k * nb + b] - ref) <= a.rel_tol * fabs(ref)) a.weights[k * nb + b] += wl / members;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = 0;
      for (int t = 0; t < nk * nb; ++t)
        if (a.weights[t] != 0.0) a.pairs[c++] = t;
      *a.npairs = c;
    }
    return;
  }
  // argmax_k lam[k][lo], lowest k among ties
  double bv = -1e300;
  int bi = 0x7fffffff;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    double v = a.lam[k * nb + lo];
    if (v > bv || (v == bv && k < bi)) { bv = v; bi = k; }
  }
  sv[threadIdx.x] = bv; si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      double v2 = sv[threadIdx.x + w]; int i2 = si[threadIdx.x + w];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) { sv[threadIdx.x] = v2; si[threadIdx.x] = i2; }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) ka_s = si[0];
  __syncthreads();
  // argmin_k lam[k][hi], lowest k among ties
  bv = 1e300; bi = 0x7fffffff;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    double v = a.lam[k * nb + hi];
    if (v < bv || (v == bv && k < bi)) { bv = v; bi = k; }
  }
  sv[threadIdx.x] = bv; si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      double v2 = sv[threadIdx.x + w]; int i2 = si[threadIdx.x + w];
      if (v2 < sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) { sv[threadIdx.x] = v2; si[threadIdx.x] = i2; }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) kb_s = si[0];
  __syncthreads();
  if (threadIdx.x != 0) return;
  int ka = ka_s, kb = kb_s;
  double la = a.lam[ka * nb + lo] * a.lref, lb = a.lam[kb * nb + hi] * a.lref;
  double G, wa, wb;
  if (a.mode == PC_GAP_OMEGA) {
    double A_ = sqrt(fmax(la, 0.0)), B_ = sqrt(fmax(lb, 0.0));
    G = 2.0 * (B_ - A_) / (B_ + A_);
    wa = A_ > 0.0 ? -2.0 * B_ / (A_ * (A_ + B_) * (A_ + B_)) : 0.0;
    wb = B_ > 0.0 ? 2.0 * A_ / (B_ * (A_ + B_) * (A_ + B_)) : 0.0;
  } else {
    G = 2.0 * (lb - la) / (lb + la);
    wa = -4.0 * lb / ((la + lb) * (la + lb));
    wb = 4.0 * la / ((la + lb) * (la + lb));
  }
  *a.gap_out = G;
  int c = 0;
  for (int side = 0; side < 2; ++side) {
    int k = side == 0 ? ka : kb;
    int band = side == 0 ? lo : hi;
    double wt = side == 0 ? wa : wb;
    double ref = a.lam[k * nb + band];
    int members = 0;
    for (int b = 0; b < nb; ++b) members += (fabs(a.lam[k * nb + b] - ref) <= a.rel_tol * fabs(ref)) ? 1 : 0;
    for (int b = 0; b < nb; ++b)
      if (fabs(a.lam[k * nb + b] - ref) <= a.rel_tol * fabs(ref)) a.weights[k * nb + b] += wt / members;
  }
  for (int t = 0; t < nk * nb; ++t)
    if (a.weights[t] != 0.0) a.pairs[c++] = t;
  *a.npairs = c;
}
int launch_gap(const GapArgs& a, cudaStream_t s) {
  k_gap<<<1, 256, 0, s>>>(a);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// ---------------------------------------------------------------------------
// Axis-2 and axis-1 synthesis of field f of pair p:
//   t2[p][f][g1][j][l] = sum_{g2,g3} c[g1][g2][g3] e^{i pi G2 (2j+1)/n1} e^{i pi G3 (2l+1)/n2}
// f < 3: displacement component f of theta; f >= 3: stress coordinate f-3.  R is the
// arithmetic of the synthesis (FP64 for the FP64 form, FP32 for the mixed form).
template <typename R>
__global__ void k_adj_synth12(AdjointArgs a) {
  typedef typename cplx_t<R>::type C2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int p = blockIdx.x, f = blockIdx.y;
  if (p >= *a.npairs) return;
  const int M2 = 2 * a.M + 1, N = a.N, n1 = a.n1, n2 = a.n2;
  C2* c = (C2*)smem;                 // N
  C2* t1 = c + N;                    // M2*M2*n2
  C2* ph3 = t1 + M2 * M2 * n2;       // M2*n2
  C2* ph2 = ph3 + M2 * n2;           // M2*n1
  const int pr = a.pairs[p];
  const int k = pr / a.nb, b = pr % a.nb;
  const long long vec = (long long)k * a.m + b;
  const long long nvec = (long long)a.nk * a.m;
  const double2* src = (f < 3) ? a.theta + (vec * 3 + f) * N : a.sig + ((long long)(f - 3) * nvec + vec) * N;
  for (int q = threadIdx.x; q < N; q += blockDim.x) c[q] = from_d2<R>(src[q]);
  for (int t = threadIdx.x; t < M2 * n2; t += blockDim.x) {
    int g = t / n2, l = t % n2;
    ph3[t] = from_d2<R>(phase_pi_over((long long)(g - a.M) * (2 * l + 1), n2));
  }
  for (int t = threadIdx.x; t < M2 * n1; t += blockDim.x) {
    int g = t / n1, j = t % n1;
    ph2[t] = from_d2<R>(phase_pi_over((long long)(g - a.M) * (2 * j + 1), n1));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < M2 * M2 * n2; t += blockDim.x) {
    int g12 = t / n2, l = t % n2;
    C2 s = mk<R>(0, 0);
    for (int g3 = 0; g3 < M2; ++g3) cfma(s, c[g12 * M2 + g3], ph3[g3 * n2 + l]);
    t1[t] = s;
  }
  __syncthreads();
  C2* out = (C2*)a.t2 + ((long long)p * 9 + f) * M2 * n1 * n2;
  for (long long t = threadIdx.x; t < (long long)M2 * n1 * n2; t += blockDim.x) {
    int l = (int)(t % n2);
    int j = (int)((t / n2) % n1);
    int g1 = (int)(t / ((long long)n1 * n2));
    C2 s = mk<R>(0, 0);
    for (int g2 = 0; g2 < M2; ++g2) cfma(s, t1[(g1 * M2 + g2) * n2 + l], ph2[g2 * n1 + j]);
    out[t] = s;
  }
}

// Axis-0 synthesis fused with the weighted reduction over (k, band).  The pairs are cut into
// chunks along the grid's z; each thread synthesises VPT voxels along axis 0 at one (j, l), so
// that every loaded axis-1/2 coefficient feeds VPT complex FMAs, and sums its chunk's three
// weighted quadratic forms in R (FP32 in the mixed form: about a hundred pairs per chunk).  The
// chunk sums go to part[chunk][3][ne]; k_adj_finish adds them in FP64 in chunk order.
constexpr int kAdjReduceThreads = 128;  // at 166 registers (M2 = 9, 4 voxels) three blocks per SM

template <typename R, int M2, int VPT>
__global__ __launch_bounds__(kAdjReduceThreads) void k_adj_reduce(AdjointArgs a, int chunk) {
  typedef typename cplx_t<R>::type C2;
  const int n0 = a.n0, n1 = a.n1, n2 = a.n2;
  const int nig = (n0 + VPT - 1) / VPT;
  const int j = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nig * n2) return;
  const int ig = v / n2, l = v % n2;
  C2 ph[VPT][M2];  // compile-time sizes and fully unrolled loops keep these in registers
#pragma unroll
  for (int s = 0; s < VPT; ++s) {
    const int i = min(ig * VPT + s, n0 - 1);
#pragma unroll
    for (int g = 0; g < M2; ++g) ph[s][g] = from_d2<R>(phase_pi_over((long long)(g - a.M) * (2 * i + 1), n0));
  }
  const int np = *a.npairs;
  const int p0 = blockIdx.z * chunk, p1 = min(np, p0 + chunk);
  const long long fstride = (long long)M2 * n1 * n2;
  const long long gstride = (long long)n1 * n2;
  const C2* t2 = (const C2*)a.t2;
  // the compliance part's factors d f1/d chi, d f2/d chi belong to the element: three weighted sums
  R acc_m[VPT], acc_1[VPT], acc_2[VPT];
#pragma unroll
  for (int s = 0; s < VPT; ++s) acc_m[s] = acc_1[s] = acc_2[s] = (R)0;
  for (int p = p0; p < p1; ++p) {
    const int pr = a.pairs[p];
    const double wd = a.weights[pr];
    const R w = (R)wd, wl = (R)(wd * a.lam[pr] * a.lref);
    const C2* base = t2 + (long long)p * 9 * fstride + (long long)j * n2 + l;
    R u2[VPT], sd[VPT], q3[VPT];
#pragma unroll
    for (int s = 0; s < VPT; ++s) u2[s] = sd[s] = q3[s] = (R)0;
#pragma unroll
    for (int f = 0; f < 9; ++f) {
      const C2* srcf = base + f * fstride;
      C2 x[M2];
#pragma unroll
      for (int g = 0; g < M2; ++g) x[g] = srcf[g * gstride];
#pragma unroll
      for (int s = 0; s < VPT; ++s) {
        C2 z = mk<R>(0, 0);
#pragma unroll
        for (int g = 0; g < M2; ++g) cfma(z, x[g], ph[s][g]);
        const R q = z.x * z.x + z.y * z.y;
        if (f < 3) u2[s] += q;
        else if (f == 3) q3[s] = q;
        else sd[s] += q;
      }
    }
#pragma unroll
    for (int s = 0; s < VPT; ++s) {
      acc_m[s] += wl * u2[s];
      acc_1[s] += w * q3[s];
      acc_2[s] += w * sd[s];
    }
  }
  const long long ne = (long long)n0 * n1 * n2;
  R* part = (R*)a.part + (long long)blockIdx.z * 3 * ne;
#pragma unroll
  for (int s = 0; s < VPT; ++s) {
    const int i = ig * VPT + s;
    if (i < n0) {
      const long long e = ((long long)i * n1 + j) * n2 + l;
      part[e] = acc_m[s];
      part[ne + e] = acc_1[s];
      part[2 * ne + e] = acc_2[s];
    }
  }
}

// The chunk sums added in FP64 and combined with the per-element factors.
template <typename R>
__global__ void k_adj_finish(AdjointArgs a, int nchunks) {
  const long long ne = (long long)a.n0 * a.n1 * a.n2;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const R* part = (const R*)a.part;
  double acc_m = 0.0, acc_1 = 0.0, acc_2 = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const R* pc = part + (long long)c * 3 * ne;
    acc_m += (double)pc[e];
    acc_1 += (double)pc[ne + e];
    acc_2 += (double)pc[2 * ne + e];
  }
  const double acc = -a.d_rho * acc_m - a.two_pi_V_sq * (a.dfc[e] * acc_1 + a.dfc[ne + e] * acc_2);
  a.grad[e] = acc * a.inv_sO * a.ve * a.dchi[e];
}

size_t adjoint_staging_bytes(int M, int n1, int n2, bool fp32) {
  const size_t M2 = 2 * (size_t)M + 1;
  const size_t elems = M2 * M2 * M2 + M2 * M2 * (size_t)n2 + M2 * (size_t)n2 + M2 * (size_t)n1;
  return elems * (fp32 ? sizeof(float2) : sizeof(double2));
}

// Voxels per thread of the reduction: 4 in FP32 (2 at M2 = 11), 1 in FP64 (register budget of
// the phase tables).
template <typename R>
constexpr int adj_vpt(int M2) { return sizeof(R) == sizeof(float) ? (M2 <= 9 ? 4 : 2) : 1; }

template <typename R>
static int launch_adjoint_t(const AdjointArgs& a, cudaStream_t s) {
  const int M2 = 2 * a.M + 1;
  if (M2 > 11) return PC_EINVAL;
  const size_t sm = adjoint_staging_bytes(a.M, a.n1, a.n2, sizeof(R) == sizeof(float));
  // Set once per instantiation; a function-local static is initialised exactly once even when
  // k groups on several host threads arrive together.
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_adj_synth12<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjointStagingMax);
  (void)attr;
  if (sm > kAdjointStagingMax) return PC_EINVAL;
  dim3 g1(a.max_pairs, 9);
  k_adj_synth12<R><<<g1, 256, sm, s>>>(a);
  PC_LAUNCH_CHECK();
  const int vpt = M2 <= 9 ? adj_vpt<R>(9) : adj_vpt<R>(11);
  const long long gx = cdiv((long long)cdiv(a.n0, vpt) * a.n2, kAdjReduceThreads);
  // enough pair chunks for about six blocks per SM; the chunks cover max_pairs, and the ones
  // past the device's pair count write zeros
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cudaGetLastError();
    return n;
  }();
  int nchunks = (int)std::min<long long>(kAdjChunksMax, std::max<long long>(1, cdiv(6LL * sms, gx * a.n1)));
  nchunks = std::max(1, std::min(nchunks, a.max_pairs));
  const int chunk = (int)cdiv(a.max_pairs, nchunks);
  nchunks = (int)cdiv(a.max_pairs, chunk);
  dim3 g2((unsigned)gx, a.n1, nchunks);
  switch (M2) {
    case 3: k_adj_reduce<R, 3, adj_vpt<R>(3)><<<g2, kAdjReduceThreads, 0, s>>>(a, chunk); break;
    case 5: k_adj_reduce<R, 5, adj_vpt<R>(5)><<<g2, kAdjReduceThreads, 0, s>>>(a, chunk); break;
    case 7: k_adj_reduce<R, 7, adj_vpt<R>(7)><<<g2, kAdjReduceThreads, 0, s>>>(a, chunk); break;
    case 9: k_adj_reduce<R, 9, adj_vpt<R>(9)><<<g2, kAdjReduceThreads, 0, s>>>(a, chunk); break;
    default: k_adj_reduce<R, 11, adj_vpt<R>(11)><<<g2, kAdjReduceThreads, 0, s>>>(a, chunk); break;
  }
  PC_LAUNCH_CHECK();
  const long long ne = (long long)a.n0 * a.n1 * a.n2;
  k_adj_finish<R><<<(unsigned)cdiv(ne, 256), 256, 0, s>>>(a, nchunks);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_adjoint(const AdjointArgs& a, bool fp32, cudaStream_t s) {
  return fp32 ? launch_adjoint_t<float>(a, s) : launch_adjoint_t<double>(a, s);
}
