/*
 * phononic.h -- C ABI of the GB300 library for mixed-variational plane-wave band
 * structures of 3-D two-phase phononic crystals and their adjoint design
 * sensitivities (Lu, Yang, Guest, Srivastava, "3-D phononic crystals with
 * ultra-wide band gaps").
 *
 * Conventions for every call below:
 *  - All pointers named *_dev are CUDA device pointers owned by the caller; *_host
 *    are host pointers owned by the caller.  The library never frees caller memory.
 *  - GPU work is enqueued asynchronously on the caller's stream (a cudaStream_t
 *    passed as void*; NULL is the legacy default stream).  Results are valid once
 *    that stream has been synchronised.
 *  - Return value: PC_OK (0) or a PC_E* code; pc_strerror() names it.  Argument
 *    errors are detected on the host before anything is enqueued.  Errors found on
 *    the device (non-convergence, bad densities, expired bounded waits) are
 *    recorded in a device status word and reported by pc_get_stats().
 *  - Every workspace is allocated by pc_create / pc_set_kpoints; pc_set_design,
 *    pc_bands and pc_gap_and_grad allocate nothing.
 *  - Units: SI.  Lattice constant a in metres, densities kg/m^3, moduli Pa.
 */
#ifndef PHONONIC_H
#define PHONONIC_H

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define PC_OK        0
#define PC_EINVAL    1  /* bad enum, size or material constant */
#define PC_EALIAS    2  /* a grid dimension n_i < 2M+1: plane waves alias on the centroids */
#define PC_ENOMEM    3  /* device allocation failed */
#define PC_ECUDA     4  /* a CUDA runtime call failed */
#define PC_ESTATE    5  /* call out of order (e.g. pc_bands before pc_set_design) */
#define PC_ENOCONV   6  /* device status: eigensolver hit max_iter for some k (outputs written) */
#define PC_EDOMAIN   7  /* device status: a density outside [0,1] or not finite */
#define PC_ETIMEOUT  8  /* device status: a bounded device-side wait expired */
#define PC_ETOOBIG   9  /* the problem exceeds the fixed working space of an allocation-free call */

/* Lattices (Methods, "Study of cubic unit cells"): primitive cells of the cubic
 * Bravais lattices, vectors along the cube edges (SC), body diagonals (BCC) and
 * face diagonals (FCC). */
#define PC_SC   0
#define PC_BCC  1
#define PC_FCC  2

/* Largest wavevector count of one context (pc_set_kpoints). */
#define PC_MAX_KPOINTS 65535

/* Material interpolation between the phases (pc_params.law). */
#define PC_LAW_COMPLIANCE 0  /* density and the compliance moduli (1-2nu)/E, (1+nu)/E linear in chi */
#define PC_LAW_YOUNG      1  /* Methods, eq. combinematerial read literally: Young's modulus and Poisson's
                                ratio linear in chi, each element the isotropic material they give */

/* Arithmetic of the eigensolver. */
#define PC_FP64   0  /* every step in FP64 on CUDA cores */
#define PC_MIXED  1  /* split-BF16 tensor-core operator, FP32 block iteration,
                        FP64 Rayleigh-Ritz and stresses at the end */

/* Degenerate clusters (pc_gap_and_grad, pc_gap_ks_and_grad): at a k-point, the bands whose
 * eigenvalue lies within this relative distance of the extremal band's share its weight equally
 * (the gradient of the cluster-mean eigenvalue, independent of the basis the solver picked inside
 * the cluster).  The FP64 form resolves eigenvalues to about 1e-12; the mixed form's final FP64
 * Rayleigh-Ritz step on FP32-converged vectors leaves symmetry-protected multiplets split by up to
 * a few 1e-8 (its eigenvalue error), so it takes a wider window. */
#define PC_CLUSTER_TOL_FP64   1e-8
#define PC_CLUSTER_TOL_MIXED  1e-6

/* Objective modes of pc_gap_and_grad. */
#define PC_GAP_OMEGA      0  /* gap = 2(b-a)/(b+a) in omega = sqrt(lambda) (Results, note on gaps) */
#define PC_GAP_LAMBDA     1  /* same in lambda = omega^2 (Methods, eq. obj) */
#define PC_GRAD_ALLBANDS  2  /* gap_dev <- sum w*lambda, grad <- sum_{k,b} w[k,b] dlambda_{k,b}/drho_e */

typedef struct pc_ctx pc_ctx;

typedef struct {
  double rho;  /* mass density, kg/m^3 (> 0) */
  double E;    /* Young's modulus, Pa (> 0) */
  double nu;   /* Poisson ratio, in (-1, 0.5) */
} pc_material;

typedef struct {
  int lattice;          /* PC_SC | PC_BCC | PC_FCC */
  double a;             /* cubic lattice constant, m (> 0) */
  int n[3];             /* voxel grid along a1, a2, a3; voxel (i,j,l) at index (i*n1+j)*n2+l */
  int M;                /* plane-wave index range -M..M per axis; N = (2M+1)^3 waves */
  pc_material phase1;   /* the phase at rho_e = 1 */
  pc_material phase0;   /* the phase at rho_e = 0 */
  double penal;         /* chi = rho^penal (>= 1); density and compliance are linear in chi */
  int nbands;           /* lowest bands returned per k: 1..24 and at most N */
  int precision;        /* PC_FP64 | PC_MIXED */
  double tol;           /* relative residual target of the block iteration (0: default, 1e-8 FP64, 3e-4 mixed).
                           A gradient through one (k, band) pair (a gap) has a relative error of
                           about that pair's final residual: for a 1e-4 gap gradient in the mixed
                           form pass tol = 1e-4 (the default suits all-band weighted objectives). */
  int max_iter;         /* iteration cap (0: default); hitting it sets PC_ENOCONV */
  int law;              /* PC_LAW_COMPLIANCE (0, default) | PC_LAW_YOUNG; density is linear in chi either way */
} pc_params;

typedef struct {
  int status;              /* first device error code seen (PC_OK if none) */
  int iterations;          /* block iterations of the last pc_bands */
  int unconverged_k;       /* k-points above tolerance when the iteration stopped */
  int nk;                  /* k-points set */
  int N;                   /* plane waves */
  int block;               /* block width m (bands + guard vectors) */
  double max_residual;     /* largest relative residual over the returned bands */
  double ms_setup;         /* last pc_set_design, device time (operator assembly) */
  double ms_bands;         /* last pc_bands, device time */
  double ms_grad;          /* last pc_gap_and_grad, device time */
  long long launches;      /* kernel launches since pc_create or the last pc_clear_status */
  /* Filled while profiling is on (pc_set_profiling), summed since it was switched on: */
  double ms_rr_gemm;       /* device time of the FP64 operator GEMMs of the Rayleigh-Ritz step */
  long long rr_gemm_launches;
  double rr_gemm_flops;    /* their algorithmic flops: 8 N^2 per complex column */
  double ms_iter_apply;    /* device time of the block iteration's operator applications */
  long long iter_apply_calls;
  double iter_apply_flops; /* algorithmic flops: 8 N^2 (6 + 3) per vector */
  double ms_small;         /* device time of the projected (small dense) problems */
  double ms_grad_kernels;  /* device time of the adjoint synthesis and reduction */
  double ms_gram;          /* device time of the block iteration's Gram products A^H B */
  long long gram_launches;
  double gram_flops;       /* algorithmic flops: 8 rows (columns of A) (columns of B) per k */
  double gram_bytes;       /* algorithmic bytes: both operands read once, the result written once */
  double ms_update;        /* device time of the block iteration's basis updates S C */
  long long update_launches;
  double update_flops;     /* algorithmic flops: 8 rows (columns of S) (columns out) per k */
  double update_bytes;     /* algorithmic bytes: inputs read once, outputs written once */
  double ms_iteration_loop; /* device time of the whole block iteration (pc_bands before its FP64 step) */
  double ms_final_rr;      /* device time of the FP64 Rayleigh-Ritz step */
  double small_flops;      /* algorithmic flops of the FP32 projected eigenproblems (mixed form) solved
                              while profiling: per problem of n coordinates, n_k kept, s Jacobi sweeps,
                              (32/3) n^3 + s n_k (n_k - 1) 12 (n_k + n) */
  long long grad_pairs;    /* weighted (k, band) pairs of the last pc_gap_and_grad / pc_gap_ks_and_grad */
  double grad_flops_per_pair; /* algorithmic flops of the adjoint per weighted pair:
                              72 ((2M+1)^3 n2 + (2M+1)^2 n1 n2 + (2M+1) n0 n1 n2) */
  double ms_host_idle;     /* stream idle time while the host reads the convergence count of each block
                              iteration and enqueues the next one (profiling; summed over the k groups) */
  int rr_sliced;           /* 1 when the Rayleigh-Ritz operator products run as exact 6-bit slice products on
                              the tensor cores (36 bf16 products per FP64-accurate one; mixed form,
                              N <= 1008), 0 when they run as the FP64 CUDA-core GEMM */
  long long small_calls;   /* calls timed in ms_small (profiling): the projected eigenproblem kernel and the
                              small Cholesky factorisations of the orthonormalisation */
} pc_stats;

/* Creates a context: validates the parameters and allocates every per-design
 * workspace (structure factors, the three N x N Toeplitz operators, the two
 * inverse compliance operators, adjoint scratch).
 * Paper: Results, eqs. mixedvariation-matrixform; Methods, eqs. loop and
 * matrixofintegral (the k-independent element-sum matrices).
 * Errors: PC_EINVAL, PC_EALIAS, PC_ENOMEM, PC_ECUDA.  *out is NULL on error. */
int pc_create(const pc_params* params, pc_ctx** out);

/* Sets the Bloch wavevectors: q_reduced_host holds nk rows of (Q1, Q2, Q3), the
 * reduced coordinates of the paper's K = T1 (Q1 + alpha) + T2 (Q2 + beta) + T3 (Q3 + gamma)
 * (reciprocal basis without 2 pi).  Allocates the block-iteration workspaces for nk
 * points (synchronous; not for use inside stream capture).  nk is at most
 * PC_MAX_KPOINTS per context; larger sets are split over several contexts.
 * Errors: PC_EINVAL (NULL, nk < 1 or nk > PC_MAX_KPOINTS), PC_ENOMEM. */
int pc_set_kpoints(pc_ctx* ctx, const double* q_reduced_host, int nk);

/* Sets the design: rho_dev holds n0*n1*n2 FP64 densities in [0, 1], C order.
 * Enqueues: SIMP interpolation (Methods, eq. combinematerial, linear in chi = rho^p),
 * structure factors of density and of the two compliance moduli at every plane-wave
 * difference (eq. loop), the Toeplitz operators (eqs. intOmega, intPhi) and the two
 * inverse compliance operators that eliminate the stress (eq. matrixform).
 * A density outside [0, 1] sets PC_EDOMAIN in the device status.
 * Errors: PC_EINVAL (NULL), PC_ECUDA. */
int pc_set_design(pc_ctx* ctx, const double* rho_dev, void* stream);

/* Band structure: omega_dev[k*nbands + b] = sqrt(max(lambda, 0)) in rad/s for the
 * lowest nbands eigenvalues of H Phi^-1 H^* U = lambda Omega U (eq. matrixform) at
 * every k, ascending.  Keeps the eigenvectors and stresses for pc_gap_and_grad.
 * Errors: PC_ESTATE (no design or no k-points), PC_EINVAL (NULL), PC_ECUDA. */
int pc_bands(pc_ctx* ctx, double* omega_dev, void* stream);

/* Normalized gap between 1-based bands n_lower and n_lower+1 over all k (Methods,
 * eq. obj; omega form by default) and its adjoint gradient (eqs. normalev,
 * sensitivityew, diffOmega, diffPhi).  gap_dev: one double.  grad_dev: n0*n1*n2
 * doubles dG/drho_e, or NULL to skip the gradient.  The max/min pick the extremal
 * (k, band); equal values at different k take the lowest k; bands within a relative
 * PC_CLUSTER_TOL_FP64 / PC_CLUSTER_TOL_MIXED of the extremal one at that k share its weight
 * equally.  For PC_GRAD_ALLBANDS,
 * w_dev holds nk*nbands weights, n_lower is ignored, gap_dev receives sum w*lambda
 * and grad_dev sum_{k,b} w[k,b] dlambda_{k,b}/drho_e.
 * The gradient stages, per CTA, the N coefficients of one field component and the
 * voxel phase tables in shared memory: N + (2M+1)^2 n2 + (2M+1)(n1 + n2) complex values
 * (16 bytes in the FP64 form, 8 in the mixed form) must fit in 200 KiB.  For cubic grids
 * n^3 that is n <= 197 / 121 / 80 (FP64) and n <= 256 / 251 / 169 (mixed) at M = 3 / 4 / 5,
 * any n <= 256 at M <= 2; larger grids get PC_EINVAL when grad_dev is given (bands and the
 * gap alone have no such limit).
 * Errors: PC_ESTATE (pc_bands not run), PC_EINVAL (n_lower out of 1..nbands-1,
 * bad mode, NULL w_dev for PC_GRAD_ALLBANDS, the grid limit above; all detected before
 * anything is enqueued), PC_ECUDA. */
int pc_gap_and_grad(pc_ctx* ctx, int n_lower, int mode, const double* w_dev,
                    double* gap_dev, double* grad_dev, void* stream);

/* Smooth surrogate of the omega-form gap between bands n_lower and n_lower+1 (not in the
 * paper, whose eq. obj takes a max and a min over k, non-differentiable where the extremal k
 * changes).  With x = omega / omega_ref, omega_ref^2 = (2 pi / a)^2 E1 / rho1 (phase 1):
 *   a = omega_ref (1/beta) log sum_k exp(beta x_{k,n}),
 *   b = -omega_ref (1/beta) log sum_k exp(-beta x_{k,n+1}),   gap = 2 (b - a) / (b + a),
 * a lower bound of the exact gap that tends to it as beta grows.  grad_dev (or NULL) receives
 * dgap/drho_e through the same adjoint as pc_gap_and_grad, with every k weighted; at each k
 * the bands within the cluster window of pc_gap_and_grad of band n (and of band n+1) share its
 * weight equally.
 * Errors: PC_ESTATE (pc_bands not run), PC_EINVAL (NULL gap_dev, n_lower out of
 * 1..nbands-1, beta not in (0, 1e12), the gradient's grid limit of pc_gap_and_grad),
 * PC_ECUDA. */
int pc_gap_ks_and_grad(pc_ctx* ctx, int n_lower, double beta, double* gap_dev, double* grad_dev, void* stream);

/* One design update of the optimization loop of Methods, eq. topopt (maximise the gap subject
 * only to xmin <= x_e <= xmax; the paper names no optimizer): a step of Svanberg's method of
 * moving asymptotes, which with bounds alone solves each variable's convex subproblem in
 * closed form.  Needs no context.  All arrays are n doubles on the device, owned by the caller:
 *   x_dev      in: the current design x^k (e.g. the densities); out: x^(k+1);
 *   df_dev     in: d(objective)/dx at x^k, of the objective being maximised (e.g. grad_dev of
 *              pc_gap_ks_and_grad);
 *   xold1_dev, xold2_dev  in: x^(k-1), x^(k-2); out: x^k, x^(k-1);
 *   low_dev, upp_dev      in: the asymptotes of the previous step; out: this step's.
 * iter = k, the number of steps taken before this one: for iter < 2 the asymptotes start at
 * x -/+ (xmax - xmin)/2 and the four history arrays are read but not used.  Later steps scale
 * the asymptote distances by 0.7 where x oscillated and by 1.2 where it kept its direction,
 * within [0.01, 10] (xmax - xmin) of x.  The new x stays within the bounds and within half the
 * box of x^k.  Non-finite gradients give non-finite designs (not checked).
 * Errors: PC_EINVAL (n < 1, a NULL array, iter < 0, xmin/xmax not finite or xmax <= xmin),
 * PC_ECUDA. */
int pc_mma_step(long long n, double* x_dev, const double* df_dev, double* xold1_dev, double* xold2_dev,
                double* low_dev, double* upp_dev, int iter, double xmin, double xmax, void* stream);

/* --- Design parametrisation (Methods, "Topology optimization formulation", the passage after
 * eq. sensitivityew; Results, "Topology optimized structures") ---
 *
 * The densities rho_e passed to pc_set_design as a closed-form function of free design
 * variables x, and the chain rule that turns d(objective)/d(rho_e) (grad_dev of pc_gap_and_grad
 * or pc_gap_ks_and_grad) into d(objective)/dx:
 *   phi   = x, or for octant = 1 (SC cells only) the image of x under the mirror symmetries
 *           a -> n_d - 1 - a of the design grid (x holds one octant, (n_d/2)^3 values);
 *   mu_e  = sum_a w_ea phi_a / sum_a w_ea over the design nodes a within `radius` of element e's
 *           centroid (Cartesian distance to the nearest periodic image), w_ea = radius - distance;
 *           design node a sits at the centre of the spacing^3 element block a (spacing 2: the
 *           paper's reduced design field with variables at twice the element size);
 *   rho_e = 1 - exp(-beta mu_e) + mu_e exp(-beta)   (Heaviside projection; beta is raised by the
 *           caller's continuation, the paper starts at beta = 1).
 * Layouts: x C-ordered over the design grid (n_i / spacing per axis) or its octant; rho over the
 * element grid n0 x n1 x n2 (the layout of pc_set_design). */
typedef struct pc_design pc_design;
typedef struct {
  int spacing;     /* design nodes every `spacing` elements along each axis: 1 or 2 */
  double radius;   /* projection radius, metres (the paper's 1.4 % of the cell is read as 1.4 element edges) */
  int octant;      /* 1: SC mirror symmetry, the free variables are one octant of the design grid */
} pc_design_params;

/* Builds the weight table of the map for the cell's lattice, a and grid n (other fields of cell
 * are not read) and allocates its device state.
 * Errors: PC_EINVAL (NULL, bad lattice or a, spacing not 1 or 2 or not dividing every n_i,
 * n_i outside 1..256, radius not positive or so large that it reaches a node's periodic image,
 * an element with no node within the radius, octant on a non-SC lattice or an odd design grid),
 * PC_ENOMEM, PC_ECUDA.  *out is NULL on error. */
int pc_design_create(const pc_params* cell, const pc_design_params* dp, pc_design** out);

/* Number of free variables (length of x), or -1 for NULL. */
long long pc_design_nvars(const pc_design* d);

/* rho_dev (n0 n1 n2 doubles) <- the densities of x_dev (nvars doubles in [0, 1]) at sharpness
 * beta > 0.  Keeps d rho / d mu of this call for pc_design_backprop.  Device pointers, stream
 * ordered.  Errors: PC_EINVAL (NULL, beta not positive and finite), PC_ECUDA. */
int pc_design_project(pc_design* d, const double* x_dev, double beta, double* rho_dev, void* stream);

/* g_x_dev (nvars doubles) <- d(objective)/dx from g_rho_dev = d(objective)/d(rho_e) (n0 n1 n2
 * doubles), at the x and beta of the last pc_design_project on this map (stream ordered after it).
 * Errors: PC_EINVAL (NULL), PC_ECUDA. */
int pc_design_backprop(pc_design* d, const double* g_rho_dev, double* g_x_dev, void* stream);

/* Frees the map.  NULL is allowed. */
void pc_design_destroy(pc_design* d);

/* --- Batches of designs of different lattices, grids and cutoffs (Methods, "Vectorization and
 * parallel computations": all wavevectors solved together) ---
 *
 * One handle over ndesigns designs, each with its own pc_params and k-points.  Every call below
 * enqueues the work of every design: a pool of `workers` host threads, each with its own
 * non-blocking stream forked from the caller's stream, drains a queue of the designs ordered by
 * estimated work (k-points x N^2, FP64 designs weighted 60x), largest first; the streams are joined
 * back to the caller's stream before the call returns, so the results are stream ordered like the
 * single-design calls.  Packed layouts, designs in order: rho and grad hold n0 n1 n2 doubles per
 * design, omega and w nk x nbands per design, gap one double per design.
 * kgroups: concurrent k groups inside each mixed-form design (0: the context default).
 * Errors of the per-design calls are returned (the first one); pc_batch_get_stats reads a design's
 * status. */
typedef struct pc_batch pc_batch;

/* params: ndesigns parameter sets; q_host: the reduced k-points of every design, concatenated
 * (nk[d] rows of 3 doubles each); workers in 1..16 (at most ndesigns are used); kgroups in 0..6.
 * Errors: PC_EINVAL (NULL, counts, any design's parameters), PC_EALIAS, PC_ENOMEM, PC_ECUDA. */
int pc_batch_create(const pc_params* params, int ndesigns, const double* q_host, const int* nk, int workers,
                    int kgroups, pc_batch** out);
/* pc_set_design of every design (rho_dev packed).  Errors: PC_EINVAL, PC_ECUDA. */
int pc_batch_set_designs(pc_batch* b, const double* rho_dev, void* stream);
/* pc_bands of every design (omega_dev packed).  Errors: PC_EINVAL, PC_ESTATE, PC_ECUDA. */
int pc_batch_bands(pc_batch* b, double* omega_dev, void* stream);
/* pc_gap_and_grad of every design: n_lower_host one value per design (ignored for
 * PC_GRAD_ALLBANDS), w_dev packed weights for PC_GRAD_ALLBANDS, gap_dev ndesigns doubles,
 * grad_dev packed or NULL.  Errors: PC_EINVAL (checked for every design before anything is
 * enqueued), PC_ESTATE, PC_ECUDA. */
int pc_batch_gap_and_grad(pc_batch* b, const int* n_lower_host, int mode, const double* w_dev, double* gap_dev,
                          double* grad_dev, void* stream);
/* pc_get_stats of one design.  Errors: PC_EINVAL (design out of range) or the design's status. */
int pc_batch_get_stats(pc_batch* b, int design, pc_stats* out);
/* Frees every design's context and the workers' streams.  NULL is allowed. */
void pc_batch_destroy(pc_batch* b);

/* Synchronises the device and fills *out; returns out->status as well. */
int pc_get_stats(pc_ctx* ctx, pc_stats* out);

/* Resets the device status word to PC_OK and the launch counter to zero. */
int pc_clear_status(pc_ctx* ctx);

/* Switches per-phase device timing on (1) or off (0); switching on zeroes the sums.
 * Timing records CUDA events on the caller's stream around the timed phases. */
int pc_set_profiling(pc_ctx* ctx, int on);

/* Measures a device throughput on the current device (synchronous, ~0.1 s):
 * what = 0: FP64 fused multiply-add rate, what = 1: FP32 fused multiply-add rate,
 * both in GFLOP/s (2 flops per FMA), with every SM busy.  Not on the hot path.
 * Errors: PC_EINVAL (bad what or NULL), PC_ECUDA. */
int pc_probe(int what, double* gflops);

/* Frees every workspace.  NULL is allowed. */
void pc_destroy(pc_ctx* ctx);

/* Static string naming a return code. */
const char* pc_strerror(int code);

/* --- Inspection entry points (used by the parity tests; not on the hot path) --- */

#define PC_EXPORT_SFAC   0  /* 3 x (4M+1)^3 complex: structure factors of rho, f1, f2 (interleaved re,im) */
#define PC_EXPORT_TOEP   1  /* 3 x N x N complex: Toeplitz operators of rho, f1, f2, SI (element sums) */
#define PC_EXPORT_WINV   2  /* 2 x N x N complex: inverses of the f1 and f2 Toeplitz operators, SI */
#define PC_EXPORT_EIGVEC 3  /* nk x nbands x 3N complex: eigenvectors, theta^H Omega theta = 1, SI */
#define PC_EXPORT_LAMBDA 4  /* nk x nbands doubles: eigenvalues lambda = omega^2, SI */
#define PC_EXPORT_WEIGHT 5  /* nk x nbands doubles: gap weights dG/dlambda of the last pc_gap_and_grad */
#define PC_EXPORT_BLOCK  6  /* nk x block x 3N complex: the final Ritz block of the last pc_bands (bands
                               and guard vectors, nondimensional; the start block pc_import_block takes) */

/* Copies an internal array to host memory (synchronous).  Returns the number of
 * doubles the array holds in *count; copies only when host != NULL and
 * capacity >= *count.  Errors: PC_EINVAL (bad which), PC_ESTATE (not computed yet). */
int pc_export(pc_ctx* ctx, int which, double* host, long long capacity, long long* count);

/* Warm start across designs (not in the paper, which solves every design from scratch): with
 * on = 1, each pc_bands starts its block iteration from the final Ritz block of the previous
 * pc_bands of this context (the bands and guard vectors of every k), when there is one for the
 * current k-points, instead of from the plane-wave start block; pc_set_kpoints discards it.  In an
 * optimization loop the next design is close to the last, so fewer iterations are needed.  The
 * results are the same eigenpairs to the iteration's tolerance.  Errors: PC_EINVAL (NULL). */
int pc_set_warm_start(pc_ctx* ctx, int on);

/* Sets the start block of the next pc_bands from host memory (count = nk x block x 3N complex
 * values as 2 count doubles, the layout of pc_export(PC_EXPORT_BLOCK), e.g. from another context
 * with the same lattice, cutoff, bands and k-points), as a warm start for that call whatever
 * pc_set_warm_start says (synchronous).  Errors: PC_EINVAL (NULL, wrong count), PC_ESTATE (no
 * k-points), PC_ECUDA. */
int pc_import_block(pc_ctx* ctx, const double* host, long long count);

/* Applies the condensed operator and the mass operator at wavevector index k to
 * ncols vectors: x_dev, ax_dev, ox_dev hold ncols x 3N complex (interleaved),
 * component-major within a vector (u1 over all waves, then u2, then u3).
 * ax = H Phi^-1 H^* x and ox = Omega x (eq. matrixform), SI units, computed with the
 * context's block-iteration operator: FP64 GEMMs for PC_FP64; for PC_MIXED, FP32
 * vectors and split-BF16 tensor-core products.  ncols <= nk * (bands + guard).
 * Requires pc_set_design and pc_set_kpoints.  Errors: PC_EINVAL, PC_ESTATE, PC_ECUDA. */
int pc_apply_operator(pc_ctx* ctx, int k, int ncols, const double* x_dev,
                      double* ax_dev, double* ox_dev, void* stream);

/* Self-check of the tensor-core kernels of the FP32 block iteration (synchronous; allocates
 * and frees its own scratch).  On seeded data with columns of norms spread over 2^-3..2^3,
 * what = 0 runs the batched Gram product G = A^H B (nblk blocks of m columns per side, n3
 * rows, nk problems) and what = 1 the basis update out = [S] C with two coefficient sets,
 * three operand triplets and an identity last block (nblk > 1), once on the split-BF16
 * tensor cores and once on the FP32 CUDA cores; *rel_err = max |difference| / max |CUDA-core
 * result|.  what = 2 exercises the failure path of the kernels' bounded barrier waits: a
 * one-thread kernel waits on a barrier that nothing completes, with a short limit; *rel_err = 0
 * when it gave up and recorded PC_ETIMEOUT and the device then accepted further work, else 1
 * (the other arguments are ignored).  what = 3 checks the FP64-accurate products of the mixed
 * form's final Rayleigh-Ritz step (exact 6-bit slices on the tensor cores) against the FP64
 * GEMM: n3 is the plane-wave count N (2N at most 2016), nk * m the columns, on seeded complex
 * data whose operator rows span eight binades.  Not on the hot path; it switches the library's Gram and
 * update kernel path for its own launches, so it must not run concurrently with other calls.
 * Errors: PC_EINVAL (m > 24,
 * nblk > 3, bad what or sizes), PC_ENOMEM, PC_ECUDA, PC_ETIMEOUT (a bounded wait of a
 * tensor-core kernel expired during what = 0 or 1). */
int pc_check_tensor_kernels(int what, int nk, int m, int nblk, int n3, double* rel_err);

/* --- Allocation-free entry point (no counterpart in the paper) ---
 *
 * For callers that may not allocate device memory once they are running: processes that
 * reserve their whole device-memory budget at start-up, loops that cannot afford the latency
 * or the implicit synchronisation of an allocation, and hosts whose allocator is not
 * available to library code.  Computes, without pc_create and without allocating, what the
 * first step of pc_set_design computes: the SIMP fields of the design and its structure
 * factors.  sfac_dev receives 3 x (4M+1)^3 complex values (interleaved re, im; density,
 * f1 = (1-2nu)/E, f2 = (1+nu)/E), the array and layout pc_export(PC_EXPORT_SFAC) returns after
 * pc_set_design.  Reads n, M, phase0, phase1 and penal from params, with the rules of pc_create
 * (the structure factors in fractional coordinates do not depend on the lattice).
 *
 * Working space: one fixed 5 MiB array in device memory, which every GPU that loads this
 * library holds until the process exits.  It fits grids up to 40^3 voxels with M <= 5;
 * larger problems are rejected with PC_ETOOBIG before anything is enqueued.
 * The first call on a device looks up that array's device address (once per device, with
 * the device current), so make the first call on each device outside any stream capture.
 * The address is kept for the life of the process: after a cudaDeviceReset of a device the
 * library must be reloaded before this entry point is used there again.
 * All calls share the array and every call overwrites it: calls that may overlap on the
 * GPU (different streams, or threads, on one device) race and must be serialised by the
 * caller.  Densities outside [0, 1] are clamped.
 * Errors: PC_EINVAL (NULL or bad parameters), PC_EALIAS, PC_ETOOBIG, PC_ECUDA. */
int pc_structure_factors_noalloc(const pc_params* params, const double* rho_dev, double* sfac_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PHONONIC_H */
