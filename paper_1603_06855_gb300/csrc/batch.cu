// Designs of different lattices, grids and cutoffs evaluated in one call (Methods, "Vectorization
// and parallel computations": every wavevector of every design is an independent problem, solved
// together).  Each design keeps its own context (operators, blocks, k-points); a call forks from
// the caller's stream, a pool of workers (host threads, one non-blocking stream each) drains a
// queue of the designs ordered by estimated work (k-points x N^2, largest first), and the workers'
// streams are joined back to the caller's stream.  The latency-bound phases of one design (the
// projected problems, the host's convergence checks) overlap the tensor- and bandwidth-bound
// phases of the others.
#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <vector>
#include "kernels.h"

struct pc_batch {
  int nd = 0;
  int workers = 1;
  std::vector<pc_ctx*> ctx;
  std::vector<pc_params> prm;
  std::vector<int> nk;
  std::vector<long long> off_rho, off_om;  // packed offsets (elements; k x bands)
  std::vector<int> order;                  // designs by estimated work, largest first
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

namespace {

// Runs fn(design, stream) for every design on the worker pool; the first error wins.
template <typename F>
int run_all(pc_batch* b, cudaStream_t caller, F fn) {
  if (cudaEventRecord(b->fork, caller) != cudaSuccess) return PC_ECUDA;
  for (int w = 0; w < b->workers; ++w)
    if (cudaStreamWaitEvent(b->streams[w], b->fork, 0) != cudaSuccess) return PC_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PC_ECUDA;
  std::atomic<int> next{0};
  std::atomic<int> err{PC_OK};
  auto work = [&](int w) {
    if (w > 0 && cudaSetDevice(dev) != cudaSuccess) { int z = PC_OK; err.compare_exchange_strong(z, PC_ECUDA); return; }
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= b->nd || err.load() != PC_OK) break;
      const int d = b->order[i];
      const int rc = fn(d, b->streams[w]);
      if (rc) { int z = PC_OK; err.compare_exchange_strong(z, rc); }
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < b->workers; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  for (int w = 0; w < b->workers; ++w) {
    if (cudaEventRecord(b->join[w], b->streams[w]) != cudaSuccess) return PC_ECUDA;
    if (cudaStreamWaitEvent(caller, b->join[w], 0) != cudaSuccess) return PC_ECUDA;
  }
  return err.load();
}

}  // namespace

extern "C" int pc_batch_create(const pc_params* params, int ndesigns, const double* q_host, const int* nk,
                               int workers, int kgroups, pc_batch** out) {
  if (!out) return PC_EINVAL;
  *out = nullptr;
  if (!params || !q_host || !nk || ndesigns < 1 || workers < 1 || workers > 16 || kgroups < 0 || kgroups > 6)
    return PC_EINVAL;
  for (int d = 0; d < ndesigns; ++d)
    if (nk[d] < 1 || nk[d] > PC_MAX_KPOINTS) return PC_EINVAL;
  pc_batch* b = new (std::nothrow) pc_batch();
  if (!b) return PC_ENOMEM;
  b->nd = ndesigns;
  b->workers = std::min(workers, ndesigns);
  b->ctx.assign(ndesigns, nullptr);
  b->prm.assign(params, params + ndesigns);
  b->nk.assign(nk, nk + ndesigns);
  b->off_rho.assign(ndesigns + 1, 0);
  b->off_om.assign(ndesigns + 1, 0);
  std::vector<double> cost(ndesigns);
  long long qoff = 0;
  int rc = PC_OK;
  for (int d = 0; d < ndesigns && rc == PC_OK; ++d) {
    const pc_params& p = params[d];
    rc = pc_create(&p, &b->ctx[d]);
    if (rc == PC_OK && kgroups > 0) rc = pc_internal_set_groups(b->ctx[d], kgroups);
    if (rc == PC_OK) rc = pc_set_kpoints(b->ctx[d], q_host + 3 * qoff, nk[d]);
    qoff += nk[d];
    b->off_rho[d + 1] = b->off_rho[d] + (long long)p.n[0] * p.n[1] * p.n[2];
    b->off_om[d + 1] = b->off_om[d] + (long long)nk[d] * p.nbands;
    const double N = (double)(2 * p.M + 1) * (2 * p.M + 1) * (2 * p.M + 1);
    cost[d] = nk[d] * N * N * (p.precision == PC_FP64 ? 60.0 : 1.0);
  }
  if (rc != PC_OK) {
    pc_batch_destroy(b);
    return rc;
  }
  b->order.resize(ndesigns);
  for (int d = 0; d < ndesigns; ++d) b->order[d] = d;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  b->streams.assign(b->workers, nullptr);
  b->join.assign(b->workers, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int w = 0; w < b->workers && ok; ++w)
    ok = cudaStreamCreateWithFlags(&b->streams[w], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[w], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pc_batch_destroy(b);
    return PC_ECUDA;
  }
  *out = b;
  return PC_OK;
}

extern "C" int pc_batch_set_designs(pc_batch* b, const double* rho_dev, void* stream) {
  if (!b || !rho_dev) return PC_EINVAL;
  return run_all(b, (cudaStream_t)stream,
                 [&](int d, cudaStream_t s) { return pc_set_design(b->ctx[d], rho_dev + b->off_rho[d], s); });
}

extern "C" int pc_batch_bands(pc_batch* b, double* omega_dev, void* stream) {
  if (!b || !omega_dev) return PC_EINVAL;
  return run_all(b, (cudaStream_t)stream,
                 [&](int d, cudaStream_t s) { return pc_bands(b->ctx[d], omega_dev + b->off_om[d], s); });
}

extern "C" int pc_batch_gap_and_grad(pc_batch* b, const int* n_lower, int mode, const double* w_dev, double* gap_dev,
                                     double* grad_dev, void* stream) {
  if (!b || !gap_dev) return PC_EINVAL;
  if (mode != PC_GAP_OMEGA && mode != PC_GAP_LAMBDA && mode != PC_GRAD_ALLBANDS) return PC_EINVAL;
  if (mode == PC_GRAD_ALLBANDS && !w_dev) return PC_EINVAL;
  if (mode != PC_GRAD_ALLBANDS) {
    if (!n_lower) return PC_EINVAL;
    for (int d = 0; d < b->nd; ++d)
      if (n_lower[d] < 1 || n_lower[d] >= b->prm[d].nbands) return PC_EINVAL;
  }
  return run_all(b, (cudaStream_t)stream, [&](int d, cudaStream_t s) {
    return pc_gap_and_grad(b->ctx[d], mode == PC_GRAD_ALLBANDS ? 1 : n_lower[d], mode,
                           w_dev ? w_dev + b->off_om[d] : nullptr, gap_dev + d,
                           grad_dev ? grad_dev + b->off_rho[d] : nullptr, s);
  });
}

extern "C" int pc_batch_get_stats(pc_batch* b, int design, pc_stats* out) {
  if (!b || !out || design < 0 || design >= b->nd) return PC_EINVAL;
  return pc_get_stats(b->ctx[design], out);
}

extern "C" void pc_batch_destroy(pc_batch* b) {
  if (!b) return;
  for (auto c : b->ctx) pc_destroy(c);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}
