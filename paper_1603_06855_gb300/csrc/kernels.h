// Internal launch interfaces shared by the translation units of the library.
#pragma once
#include "common.cuh"

// A phase accepted by pc_create: rho > 0, E > 0 (both finite), -1 < nu < 0.5.
bool pc_material_ok(const pc_material& m);
// Concurrent k groups of a context's mixed form, set before pc_set_kpoints (phononic.cu).
int pc_internal_set_groups(pc_ctx* c, int groups);

struct MaterialConsts {
  int law;             // PC_LAW_COMPLIANCE | PC_LAW_YOUNG
  double E0, E1, nu0, nu1;  // Young's modulus and Poisson ratio of phase0 / phase1 (PC_LAW_YOUNG)
  double penal;
  double rho0, rho1;   // mass density of phase0 / phase1
  double f1_0, f1_1;   // bulk compliance (1-2nu)/E
  double f2_0, f2_1;   // shear compliance (1+nu)/E
};

struct SetupArgs {
  const double* rho;
  int n0, n1, n2, M;
  double V;
  MaterialConsts mc;
  double* fields;   // 3 x ne
  double* dchi;     // ne
  double* chi;      // ne
  double* dfc;      // 2 x ne: d f1 / d chi, d f2 / d chi per element
  double* chi_mean; // 1
  double2* t1;      // 3 x n0 x n1 x L
  double2* t2;      // 3 x n0 x L x L
  double2* sfac;    // 3 x L^3
  double2* T;       // 3 x N x N   (density, f1, f2), SI
  double2* W;       // 2 x N x N   inverses of the f1, f2 blocks, SI
  double2* gj_row;  // 2 panels x 2 x 32 x N: old pivot rows of the blocked Gauss-Jordan steps
  double2* gj_col;  // 2 panels x 2 x 32 x (N + 32): pivot-block inverses and column panels
  int* status;
  cudaStream_t side;       // stream for the next panel's pivot block (or null: one stream)
  cudaEvent_t ev_rows;     // the next pivot's rows are updated
  cudaEvent_t ev_pivot;    // the next pivot block is inverted
};
int launch_setup(const SetupArgs& a, cudaStream_t s);

// Geometry needed on the device to form K_q = T (Q_k + g_q).
struct Geom {
  double T[9];  // reciprocal basis, row-major: K_i = sum_j T[i*3+j] * (Q_j + g_j)
  int M;
  int N;
};

// Complex GEMM C[col][p] = alpha * sum_q A[p][q] B[col][q]   (both operands K-contiguous)
template <typename R>
int launch_gemm(int Mrows, int ncols, int K, const typename cplx_t<R>::type* A, int lda,
                const typename cplx_t<R>::type* B, long long ldb, typename cplx_t<R>::type* C,
                long long ldc, R alpha, cudaStream_t s);

// Operator pieces.  Vector blocks are [vec][3][N] complex, vec = k*m + j.
template <typename R>
int launch_strain(const typename cplx_t<R>::type* X, int nvec, int m, Geom g, const double* Q,
                  typename cplx_t<R>::type* E, cudaStream_t s, const float4* Kf = nullptr);
template <typename R>
int launch_epilogue(const typename cplx_t<R>::type* Sig, int nvec, int m, Geom g, const double* Q,
                    R c0, R c1, typename cplx_t<R>::type* AX, cudaStream_t s, const float4* Kf = nullptr);
// Kf[k N + q] = FP32 wavevector (K_0, K_1, K_2, 0) of plane wave q at the k-th point of Q (nk points);
// the FP32 kernels above and below read it when given (it is ignored for FP64 data).
int launch_kvec_table(Geom g, const double* Q, int nk, float4* Kf, cudaStream_t s);

struct PrecConsts {
  double c_mu;    // (2pi)^2 V mu_ref / sA ... multiplied by |K|^2
  double c_lm;    // (2pi)^2 V (lambda_ref + mu_ref) / sA
  double c_rho;   // 0.5 * lambda_scale * V rho_ref / sA
};
struct PrecRef {  // reference medium from the mean of chi (device scalar)
  double lam0, lam1, mu0, mu1, rho0, rho1;
  double f1_0, f1_1, f2_0, f2_1;  // compliance moduli (1-2nu)/E, (1+nu)/E of the phases
  double two_pi_sq_V_over_sA;
  double half_lref_V_over_sA;
  int ref_mode;       // 0: Lame constants linear in chi; 1: compliance linear in chi (the material law)
  double shift_scale; // weight of the mass term rho sigma
};
template <typename R>
int launch_resnorm(const typename cplx_t<R>::type* AX, const typename cplx_t<R>::type* OX,
                   const R* lam, int nk, int m, int nb, int n3, double tol, double* rnorm,
                   int* active, int* kdone, int* unconv, cudaStream_t s, double* best = nullptr,
                   int* since = nullptr);
template <typename R>
int launch_precond(const typename cplx_t<R>::type* AX, const typename cplx_t<R>::type* OX,
                   const R* lam, const int* active, const int* kdone, int nk, int m, int nb, Geom g,
                   const double* Q, PrecRef pr, const double* chi_mean, typename cplx_t<R>::type* W, cudaStream_t s,
                   const float4* Kf = nullptr);
template <typename R>
int launch_init_guess(typename cplx_t<R>::type* X, int nk, int m, Geom g, const double* Q, unsigned long long seed,
                      cudaStream_t s);

// Block operations of the eigensolver, batched over k.  A "block" is m vectors of n3 rows
// per k, base pointer + k * m * n3.
template <typename R> struct BlockList {
  const typename cplx_t<R>::type* p[3];
};
template <typename R>
int launch_gram(BlockList<R> A, int na, BlockList<R> B, int nb_, int nk, int m, int n3, R scale,
                typename cplx_t<R>::type* part, typename cplx_t<R>::type* G, cudaStream_t s, int* status = nullptr);
template <typename R> struct UpdateArgs {
  const typename cplx_t<R>::type* in[3][3];  // [triplet][block]
  typename cplx_t<R>::type* out[3];
  int ntrip, nblk;
  int identity_last;   // out = in[last] + sum_{b<last} in[b] C_b
  const typename cplx_t<R>::type* C;  // per k: rows (nblk or nblk-1)*m, cols mout
  long long cstride;   // elements per k in C
  int cld;             // leading dimension (columns) of C
  int m, mout, n3, nk;
  long long in_kstride, out_kstride;  // elements per k (normally m*n3 / mout*n3)
  // optional second coefficient set over the same inputs: out2[t] = sum_b in[t][b] C2nd_b
  const typename cplx_t<R>::type* C2nd = nullptr;
  typename cplx_t<R>::type* out2[3] = {nullptr, nullptr, nullptr};
  int* status = nullptr;  // device status word (tensor-core kernels record a timeout there)
};
template <typename R> int launch_update(const UpdateArgs<R>& a, cudaStream_t s);
// Tensor-core versions for FP32 data (tall_tc.cu); g_tc_tall = 0 selects the CUDA-core kernels.
// Process-wide switches read by every launch, from any k-group thread.
extern std::atomic<int> g_tc_tall;
int launch_gram_tc(const float2* const A[3], int na, const float2* const B[3], int nbk, int nk, int m, int n3,
                   float scale, float2* part, int max_split, float2* G, int* status, cudaStream_t s);
int launch_update_tc(const UpdateArgs<float>& u, int* status, cudaStream_t s);

template <typename R>
int launch_small_rr(const typename cplx_t<R>::type* GA, const typename cplx_t<R>::type* GO, int n, int m,
                    int nk, R drop_tol, const int* kdone, R* lam_out, typename cplx_t<R>::type* coef, int* status,
                    cudaStream_t s);
// The FP32 projected problems of the mixed form (small_rr.cu): same contract as
// launch_small_rr<float>; when cp is given, the conjugate-direction coefficients of
// launch_small_pdir<float> (absolute drop level pdir_abs) are computed by the same CTAs; when
// flops is given, the algorithmic flops of every problem solved are added to it (device counter).
int launch_small_rr32(const float2* GA, const float2* GO, int n, int m, int nk, float drop_tol, const int* kdone,
                      float* lam_out, float2* coef, float2* cp, float pdir_abs, int* status, double* flops,
                      cudaStream_t s);
// Cholesky-QR transform of the Gram G (m x m per k).  When Gref is given (rows_ref x m per
// k, scale -1, its last m rows holding -Y^H Omega Y before projection), a column whose
// Omega-norm^2 after projection is below rel_tol times the one before is dropped.
template <typename R>
int launch_small_chol(const typename cplx_t<R>::type* G, int m, int nk, R drop_tol,
                      const typename cplx_t<R>::type* Gref, int rows_ref, R rel_tol,
                      typename cplx_t<R>::type* T, cudaStream_t s);

// Conjugate-direction coefficients from the Ritz coefficients (see lobpcg.cu).
template <typename R>
int launch_small_pdir(const typename cplx_t<R>::type* GO, const typename cplx_t<R>::type* CX, int n, int m, int nk,
                      const int* kdone, R abs_drop, typename cplx_t<R>::type* CP, cudaStream_t s);

int launch_convert_f2d(const float2* src, double2* dst, long long n, cudaStream_t s);

// Gap objective and adjoint.
struct GapArgs {
  const double* lam;     // nk x nb, nondimensional
  int nk, nb, n_lower, mode;
  double lref;           // lambda_phys = lam * lref
  double rel_tol;
  double ks_beta;        // smooth (KS) gap: sharpness on omega / omega_ref (mode PC_GAP_KS_INTERNAL)
  const double* w_user;  // for PC_GRAD_ALLBANDS
  double* gap_out;
  double* weights;       // nk x nb, dG / dlambda_phys
  int* pairs;            // list of (k*nb + b) with non-zero weight
  int* npairs;
};
int launch_gap(const GapArgs& a, cudaStream_t s);
#define PC_GAP_KS_INTERNAL 3  // mode of GapArgs for pc_gap_ks_and_grad

struct AdjointArgs {
  const double2* theta;  // [vec][3][N], nondimensional eigenvectors (X' with X'^H Omega' X' = I)
  const double2* sig;    // [6][nvec][N], W_s E_s of theta (SI W, strain without 2 pi)
  const double* lam;     // nk x nb nondimensional
  const double* weights; // nk x nb physical
  const int* pairs;
  const int* npairs;
  int max_pairs;
  int nk, nb, m, N, M, n0, n1, n2;
  double lref;           // physical lambda scale
  double inv_sO;         // |theta_phys|^2 = |X'|^2 / sO
  double d_rho;
  const double* dfc;     // 2 x ne: d f1 / d chi and d f2 / d chi per element
  double two_pi_V_sq;    // (2 pi V)^2
  double ve;             // element volume
  const double* dchi;
  void* t2;              // scratch: max_pairs x 9 x M2 x n1 x n2 complex (FP64 or FP32)
  void* part;            // scratch: kAdjChunksMax x 3 x ne chunk sums (FP64 or FP32)
  double* grad;
};
constexpr int kAdjChunksMax = 32;  // pair chunks of the adjoint's reduction
// fp32: synthesis in FP32 (mixed form); the weighted sum is accumulated in FP64 either way.
int launch_adjoint(const AdjointArgs& a, bool fp32, cudaStream_t s);
// Dynamic shared memory of the adjoint's field-synthesis kernel: the N coefficients of one
// eigenvector component plus the (2M+1)^2 n2 and (2M+1)(n1 + n2) phase tables, complex values
// of the form's precision.  Grids and cutoffs above kAdjointStagingMax are refused.
size_t adjoint_staging_bytes(int M, int n1, int n2, bool fp32);
constexpr size_t kAdjointStagingMax = 200 * 1024;

// omega[k][b] = sqrt(max(lam_m[k][b] * lref, 0)) and lam_nd[k][b] = lam_m[k][b] for b < nb.
int launch_omega(const double* lam_m, int nk, int nb, int m, double lref, double* omega, double* lam_nd,
                 cudaStream_t s);
int launch_d2f(const double2* src, float2* dst, long long n, double scale, cudaStream_t s);
int launch_scale_d2(double2* x, long long n, double s, cudaStream_t st);
