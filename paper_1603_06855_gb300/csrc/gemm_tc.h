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
int tc_apply(TcPlan* p, const float2* X, float2* AX, float2* OX, int nvec, int m, Geom g, const double* Q, cudaStream_t s);
