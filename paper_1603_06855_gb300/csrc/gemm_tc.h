// Split-BF16 tensor-core (tcgen05) operator application for the mixed-precision path.
#pragma once
#include "kernels.h"

struct TcPlan;
// status: device word that receives PC_ETIMEOUT if a bounded wait expires.
TcPlan* tc_plan_create(int N, int nvec, int* status);
// A plan with its own vector workspaces (capacity nvec) that applies the operators prepared in
// `ops` (which must outlive it); for k-point subsets run concurrently on separate streams.
TcPlan* tc_plan_create_sharing(const TcPlan* ops, int nvec, int* status);
void tc_plan_destroy(TcPlan* p);
bool tc_available(const TcPlan* p);
// Converts the FP64 operators (W1, W2 in SI; T_rho in SI) into the scaled split-BF16
// tensor-core operands: W * w_scale and T_rho * t_scale.
int tc_prepare_operators(TcPlan* p, const double2* W, const double2* T, double w_scale, double t_scale, cudaStream_t s);
// AX, OX for nvec FP32 vectors (vector v at k = v / m).
int tc_apply(TcPlan* p, const float2* X, float2* AX, float2* OX, int nvec, int m, Geom g, const double* Q, cudaStream_t s,
             const float4* Kf = nullptr);

// FP64-accurate operator products by exact 6-bit slicing on the tensor cores (oz_gemm.cu), for
// the mixed form's final Rayleigh-Ritz step.  Eligible for 2N (padded to 32) below 2048.
struct OzPlan;
bool oz_eligible(int N);
// ncap: right-hand-side columns the plan holds; share: a plan whose operator slices to use.
OzPlan* oz_plan_create(int N, int ncap, int* status, const OzPlan* share);
void oz_plan_destroy(OzPlan* p);
bool oz_available(const OzPlan* p);
// Slices of W1 * w_scale, W2 * w_scale, T_rho * t_scale (complex N x N, FP64).
int oz_prepare_operators(OzPlan* p, const double2* W, const double2* T, double w_scale, double t_scale, cudaStream_t s);
// Slices of ncols complex FP64 columns of length N into right-hand-side columns col_off..
int oz_slice_columns(OzPlan* p, const double2* X, int ncols, int col_off, cudaStream_t s);
// C (ncols complex columns of length N) = operator which_A (0: W1, 1: W2, 2: T_rho) times the
// right-hand-side columns col_base..col_base + ncols.
int oz_gemm(OzPlan* p, int which_A, int col_base, int ncols, double2* C, cudaStream_t s);
// max |sliced - FP64| / max |FP64| on seeded data (N waves, ncols columns).
int oz_self_check(int N, int ncols, double* rel_err);
