// Allocation-free structure factors.
//
// Some callers cannot allocate device memory while they run: a host that has reserved all
// of its device memory up front and forbids further cudaMalloc (a long-running service or a
// memory-budgeted job), code that must not add allocation latency or implicit device
// synchronisation to a time-critical loop, or a caller that drives the library from a
// context where the allocator is simply unavailable.  pc_structure_factors_noalloc gives
// them the SIMP fields and the three structure factors of a design without pc_create: its
// working space is the file-scope array below, which every device that loads this library
// holds until the process exits.
#include <cmath>
#include <mutex>
#include "kernels.h"

// Working space of the allocation-free path: SIMP fields (3 ne), chi and dchi (2 ne), and the
// two partial-sum stages of the separable sums (3 n0 n1 L and 3 n0 L^2 complex), for grids up
// to 40^3 and cutoffs up to M = 5 (L = 4M + 1 = 21): 5 MiB.
#define PC_NOALLOC_BYTES (5u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[PC_NOALLOC_BYTES];

// Kernels of the structure-factor step (defined in setup.cu).
__global__ void k_interp(const double* __restrict__ rho, int ne, MaterialConsts mc, double* __restrict__ fields,
                         double* __restrict__ dchi, double* __restrict__ chi_out, int* status, double* dfc);
__global__ void k_sfac1(const double* __restrict__ fields, int n0, int n1, int n2, int M, double2* __restrict__ t1);
__global__ void k_sfac2(const double2* __restrict__ t1, int n0, int n1, int M, double2* __restrict__ t2);
__global__ void k_sfac3(const double2* __restrict__ t2, int n0, int M, double inv_ne, double2* __restrict__ sf);

namespace {
const int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;  // calls from several host threads look the address up once

// Device address of the scratch array on the current device, looked up once per device (the
// set-up step of the first call there).  A cudaDeviceReset destroys the module that holds the
// array, so the recorded address is stale afterwards; the header says so.
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PC_ECUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PC_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_ptr[dev];
  return PC_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

extern "C" int pc_structure_factors_noalloc(const pc_params* p, const double* rho_dev, double* sfac_dev,
                                            void* stream) {
  // the same parameter rules as pc_create (the lattice and the band fields are not read)
  if (!p || !rho_dev || !sfac_dev) return PC_EINVAL;
  if (p->M < 1 || p->M > 5) return PC_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (p->n[i] < 1 || p->n[i] > 256) return PC_EINVAL;
  if (!pc_material_ok(p->phase0) || !pc_material_ok(p->phase1)) return PC_EINVAL;
  if (!(p->penal >= 1.0) || !std::isfinite(p->penal)) return PC_EINVAL;
  if (p->law != PC_LAW_COMPLIANCE && p->law != PC_LAW_YOUNG) return PC_EINVAL;
  const int M2 = 2 * p->M + 1;
  for (int i = 0; i < 3; ++i)
    if (p->n[i] < M2) return PC_EALIAS;
  const int n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
  const long long ne = (long long)n0 * n1 * n2;
  const int L = 4 * p->M + 1;
  // carve the scratch array; reject anything that does not fit
  const size_t b_fields = align256(sizeof(double) * 3 * ne);
  const size_t b_chi = align256(sizeof(double) * ne);
  const size_t b_t1 = align256(sizeof(double2) * 3 * (size_t)n0 * n1 * L);
  const size_t b_t2 = align256(sizeof(double2) * 3 * (size_t)n0 * L * L);
  const size_t b_status = 256;
  if (b_fields + 2 * b_chi + b_t1 + b_t2 + b_status > PC_NOALLOC_BYTES) return PC_ETOOBIG;
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  double* fields = (double*)base;
  double* dchi = (double*)(base + b_fields);
  double* chi = (double*)(base + b_fields + b_chi);
  double2* t1 = (double2*)(base + b_fields + 2 * b_chi);
  double2* t2 = (double2*)(base + b_fields + 2 * b_chi + b_t1);
  int* status = (int*)(base + b_fields + 2 * b_chi + b_t1 + b_t2);

  cudaStream_t s = (cudaStream_t)stream;
  cudaGetLastError();
  MaterialConsts mc;
  mc.law = p->law;
  mc.E0 = p->phase0.E;
  mc.E1 = p->phase1.E;
  mc.nu0 = p->phase0.nu;
  mc.nu1 = p->phase1.nu;
  mc.penal = p->penal;
  mc.rho0 = p->phase0.rho;
  mc.rho1 = p->phase1.rho;
  mc.f1_0 = (1.0 - 2.0 * p->phase0.nu) / p->phase0.E;
  mc.f1_1 = (1.0 - 2.0 * p->phase1.nu) / p->phase1.E;
  mc.f2_0 = (1.0 + p->phase0.nu) / p->phase0.E;
  mc.f2_1 = (1.0 + p->phase1.nu) / p->phase1.E;
  // the status word is the only part read before written: clear it for this call
  PC_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
  k_interp<<<cdiv(ne, 256), 256, 0, s>>>(rho_dev, (int)ne, mc, fields, dchi, chi, status, nullptr);
  PC_LAUNCH_CHECK();
  const long long t1n = 3LL * n0 * n1 * L;
  k_sfac1<<<cdiv(t1n, 256), 256, 0, s>>>(fields, n0, n1, n2, p->M, t1);
  PC_LAUNCH_CHECK();
  const long long t2n = 3LL * n0 * L * L;
  k_sfac2<<<cdiv(t2n, 256), 256, 0, s>>>(t1, n0, n1, p->M, t2);
  PC_LAUNCH_CHECK();
  const long long sfn = 3LL * L * L * L;
  k_sfac3<<<cdiv(sfn, 256), 256, 0, s>>>(t2, n0, p->M, 1.0 / (double)ne, (double2*)sfac_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
