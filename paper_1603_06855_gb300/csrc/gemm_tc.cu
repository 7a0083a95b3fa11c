#include "gemm_tc.h"
struct TcPlan { int N, nvec; };
TcPlan* tc_plan_create(int N, int nvec) { TcPlan* p = new TcPlan; p->N = N; p->nvec = nvec; return p; }
void tc_plan_destroy(TcPlan* p) { delete p; }
bool tc_available(const TcPlan*) { return false; }
int tc_prepare_operators(TcPlan*, const double2*, const double2*, double, double, cudaStream_t) { return PC_OK; }
int tc_apply(TcPlan*, const float2*, float2*, float2*, int, int, Geom, const double*, cudaStream_t) { return PC_EINVAL; }
