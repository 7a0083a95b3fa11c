// Design parametrisation (Methods, "Topology optimization formulation", the passage after eq.
// sensitivityew; Results, "Topology optimized structures"): element densities as a closed-form
// function of a reduced design field, and the chain rule back.
//
//   x (free variables) --[SC octant mirror, optional]--> phi (design nodes, every `spacing`
//   elements) --[linear-weight average within the radius]--> mu (elements)
//   --[Heaviside projection]--> rho_e = 1 - exp(-beta mu_e) + mu_e exp(-beta)
//
// Design node a of a spacing-2 grid sits at the centre of the 2 x 2 x 2 element block a,
// fractional position (2a + 1) / n per axis; with spacing 1 the nodes are the element centroids.
// Element e averages the nodes within the radius r with weights w = r - |x_a - x_e| (Cartesian,
// nearest periodic image).  The weight of a node depends only on its offset d (in nodes) from the
// element's block and on the element's position p inside its block (its parity class), so one
// table of (p, d, w) serves every element (forward: gather over the nodes of the element's class)
// and every node (backward: gather over the elements e = spacing (a - d) + p of each class).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>
#include "kernels.h"

struct DesignEntry {
  int d0, d1, d2;  // node offset from the element's block
  double w;        // weight / total weight of the class
};

struct pc_design {
  int n[3], nd[3], spacing, octant;
  long long ne, nnodes, nvars;
  int nclass;
  DesignEntry* table = nullptr;  // device: entries of class 0, then class 1, ...
  int* class_start = nullptr;    // device: nclass + 1 offsets into table
  double* phi = nullptr;         // device: nnodes, the expanded design field (octant maps)
  double* gphi = nullptr;        // device: nnodes, dG/dphi before folding
  double* dmu = nullptr;         // device: ne, d rho / d mu of the last projection
};

namespace {

__global__ void k_octant_expand(const double* __restrict__ x, int nd0, int nd1, int nd2, double* __restrict__ phi) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nn = (long long)nd0 * nd1 * nd2;
  if (t >= nn) return;
  const int l = (int)(t % nd2), j = (int)((t / nd2) % nd1), i = (int)(t / ((long long)nd1 * nd2));
  const int h1 = nd1 / 2, h2 = nd2 / 2;
  const int a = min(i, nd0 - 1 - i), b = min(j, nd1 - 1 - j), c = min(l, nd2 - 1 - l);
  phi[t] = x[((long long)a * h1 + b) * h2 + c];
}

// Adjoint of the expansion: each octant variable sums the gradient of its 8 images.
__global__ void k_octant_fold(const double* __restrict__ g, int nd0, int nd1, int nd2, double* __restrict__ gx) {
  const int h0 = nd0 / 2, h1 = nd1 / 2, h2 = nd2 / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)h0 * h1 * h2) return;
  const int c = (int)(t % h2), b = (int)((t / h2) % h1), a = (int)(t / ((long long)h1 * h2));
  double s = 0.0;
  for (int m = 0; m < 8; ++m) {
    const int i = (m & 1) ? nd0 - 1 - a : a, j = (m & 2) ? nd1 - 1 - b : b, l = (m & 4) ? nd2 - 1 - c : c;
    s += g[((long long)i * nd1 + j) * nd2 + l];
  }
  gx[t] = s;
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__global__ void k_project(const double* __restrict__ phi, const DesignEntry* __restrict__ tab,
                          const int* __restrict__ cstart, int n0, int n1, int n2, int nd0, int nd1, int nd2, int sp,
                          double beta, double* __restrict__ rho, double* __restrict__ dmu) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n0 * n1 * n2) return;
  const int l = (int)(e % n2), j = (int)((e / n2) % n1), i = (int)(e / ((long long)n1 * n2));
  const int b0 = i / sp, b1 = j / sp, b2 = l / sp;
  const int p = ((i - b0 * sp) * sp + (j - b1 * sp)) * sp + (l - b2 * sp);
  double mu = 0.0;
  for (int q = cstart[p]; q < cstart[p + 1]; ++q) {
    const DesignEntry t = tab[q];
    const int a0 = wrap(b0 + t.d0, nd0), a1 = wrap(b1 + t.d1, nd1), a2 = wrap(b2 + t.d2, nd2);
    mu += t.w * phi[((long long)a0 * nd1 + a1) * nd2 + a2];
  }
  // mu is a convex combination of values in [0, 1]: the clamps only remove rounding excursions
  // (a density 1 ulp above 1 would be flagged PC_EDOMAIN by pc_set_design)
  mu = fmin(fmax(mu, 0.0), 1.0);
  const double em = exp(-beta * mu), eb = exp(-beta);
  rho[e] = fmin(fmax(1.0 - em + mu * eb, 0.0), 1.0);
  dmu[e] = beta * em + eb;
}

// dG/dphi_a = sum over the elements e that average node a of w_ea dG/drho_e drho_e/dmu_e.
__global__ void k_project_grad(const double* __restrict__ g_rho, const double* __restrict__ dmu,
                               const DesignEntry* __restrict__ tab, const int* __restrict__ cstart, int nclass,
                               int n1, int n2, int nd0, int nd1, int nd2, int sp, double* __restrict__ gphi) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= (long long)nd0 * nd1 * nd2) return;
  const int a2 = (int)(a % nd2), a1 = (int)((a / nd2) % nd1), a0 = (int)(a / ((long long)nd1 * nd2));
  double s = 0.0;
  for (int p = 0; p < nclass; ++p) {
    const int p0 = p / (sp * sp), p1 = (p / sp) % sp, p2 = p % sp;
    for (int q = cstart[p]; q < cstart[p + 1]; ++q) {
      const DesignEntry t = tab[q];
      const int b0 = wrap(a0 - t.d0, nd0), b1 = wrap(a1 - t.d1, nd1), b2 = wrap(a2 - t.d2, nd2);
      const long long e = ((long long)(sp * b0 + p0) * n1 + (sp * b1 + p1)) * n2 + (sp * b2 + p2);
      s += t.w * g_rho[e] * dmu[e];
    }
  }
  gphi[a] = s;
}

void lattice_columns(int lat, double a, double A[9]) {
  // columns a_1, a_2, a_3 (A[r*3+c] = component r of a_c)
  static const double P[3][3][3] = {{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
                                    {{-0.5, 0.5, 0.5}, {0.5, -0.5, 0.5}, {0.5, 0.5, -0.5}},
                                    {{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}}};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[r * 3 + c] = a * P[lat][c][r];
}

}  // namespace

extern "C" int pc_design_create(const pc_params* cell, const pc_design_params* dp, pc_design** out) {
  if (!out) return PC_EINVAL;
  *out = nullptr;
  if (!cell || !dp) return PC_EINVAL;
  if (cell->lattice < PC_SC || cell->lattice > PC_FCC || !(cell->a > 0) || !std::isfinite(cell->a)) return PC_EINVAL;
  if (dp->spacing != 1 && dp->spacing != 2) return PC_EINVAL;
  if (!(dp->radius > 0) || !std::isfinite(dp->radius)) return PC_EINVAL;
  if (dp->octant != 0 && dp->octant != 1) return PC_EINVAL;
  if (dp->octant && cell->lattice != PC_SC) return PC_EINVAL;
  const int sp = dp->spacing;
  int n[3], nd[3];
  for (int i = 0; i < 3; ++i) {
    n[i] = cell->n[i];
    if (n[i] < 1 || n[i] > 256 || n[i] % sp) return PC_EINVAL;
    nd[i] = n[i] / sp;
    if (dp->octant && nd[i] % 2) return PC_EINVAL;
  }
  double A[9];
  lattice_columns(cell->lattice, cell->a, A);
  // reciprocal vectors b_i (rows of A^-1).  A node at offset d along axis i has fractional offset
  // f_i = (sp d + sp/2 - p_i - 1/2) / n_i from the element and lies at least |f_i| / |b_i| away, so
  // only |sp d| < r n_i |b_i| + (sp - 1)/2 can fall within the radius: |d| <= R_i below.
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                         (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                         (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                         (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                         (A[0] * A[4] - A[1] * A[3]) / det};
  int R[3];
  for (int i = 0; i < 3; ++i) {
    const double bl = std::sqrt(inv[i * 3] * inv[i * 3] + inv[i * 3 + 1] * inv[i * 3 + 1] + inv[i * 3 + 2] * inv[i * 3 + 2]);
    R[i] = (int)std::floor((dp->radius * n[i] * bl + 0.5 * (sp - 1)) / sp);
    if (2 * R[i] + 1 > nd[i]) return PC_EINVAL;  // the radius reaches a node's periodic image
  }
  // weight table per parity class
  const int nclass = sp * sp * sp;
  std::vector<DesignEntry> tab;
  std::vector<int> cstart(nclass + 1, 0);
  for (int p = 0; p < nclass; ++p) {
    const int pc[3] = {p / (sp * sp), (p / sp) % sp, p % sp};
    const size_t first = tab.size();
    double tot = 0.0;
    for (int d0 = -R[0]; d0 <= R[0]; ++d0)
      for (int d1 = -R[1]; d1 <= R[1]; ++d1)
        for (int d2 = -R[2]; d2 <= R[2]; ++d2) {
          const int d[3] = {d0, d1, d2};
          double best = 1e300;
          for (int s0 = -1; s0 <= 1; ++s0)
            for (int s1 = -1; s1 <= 1; ++s1)
              for (int s2 = -1; s2 <= 1; ++s2) {
                const int sh[3] = {s0, s1, s2};
                double f[3], x[3] = {0, 0, 0};
                for (int ax = 0; ax < 3; ++ax) f[ax] = (sp * d[ax] + 0.5 * sp - pc[ax] - 0.5) / n[ax] + sh[ax];
                for (int r = 0; r < 3; ++r)
                  for (int c = 0; c < 3; ++c) x[r] += A[r * 3 + c] * f[c];
                best = std::fmin(best, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
              }
          const double w = dp->radius - best;
          if (w > 0) {
            tab.push_back(DesignEntry{d0, d1, d2, w});
            tot += w;
          }
        }
    if (!(tot > 0)) return PC_EINVAL;  // an element sees no node within the radius
    for (size_t q = first; q < tab.size(); ++q) tab[q].w /= tot;
    cstart[p + 1] = (int)tab.size();
  }
  pc_design* d = new (std::nothrow) pc_design();
  if (!d) return PC_ENOMEM;
  memcpy(d->n, n, sizeof(n));
  memcpy(d->nd, nd, sizeof(nd));
  d->spacing = sp;
  d->octant = dp->octant;
  d->ne = (long long)n[0] * n[1] * n[2];
  d->nnodes = (long long)nd[0] * nd[1] * nd[2];
  d->nvars = dp->octant ? d->nnodes / 8 : d->nnodes;
  d->nclass = nclass;
  bool ok = cudaMalloc(&d->table, sizeof(DesignEntry) * tab.size()) == cudaSuccess &&
            cudaMalloc(&d->class_start, sizeof(int) * (nclass + 1)) == cudaSuccess &&
            cudaMalloc(&d->phi, sizeof(double) * d->nnodes) == cudaSuccess &&
            cudaMalloc(&d->gphi, sizeof(double) * d->nnodes) == cudaSuccess &&
            cudaMalloc(&d->dmu, sizeof(double) * d->ne) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pc_design_destroy(d);
    return PC_ENOMEM;
  }
  if (cudaMemcpy(d->table, tab.data(), sizeof(DesignEntry) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d->class_start, cstart.data(), sizeof(int) * (nclass + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d->dmu, 0, sizeof(double) * d->ne) != cudaSuccess) {
    pc_design_destroy(d);
    return PC_ECUDA;
  }
  *out = d;
  return PC_OK;
}

extern "C" long long pc_design_nvars(const pc_design* d) { return d ? d->nvars : -1; }

extern "C" int pc_design_project(pc_design* d, const double* x, double beta, double* rho, void* stream) {
  if (!d || !x || !rho || !(beta > 0) || !std::isfinite(beta)) return PC_EINVAL;
  cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  const double* phi = x;
  if (d->octant) {
    k_octant_expand<<<cdiv(d->nnodes, 256), 256, 0, s>>>(x, d->nd[0], d->nd[1], d->nd[2], d->phi);
    PC_LAUNCH_CHECK();
    phi = d->phi;
  }
  k_project<<<cdiv(d->ne, 256), 256, 0, s>>>(phi, d->table, d->class_start, d->n[0], d->n[1], d->n[2], d->nd[0],
                                             d->nd[1], d->nd[2], d->spacing, beta, rho, d->dmu);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

extern "C" int pc_design_backprop(pc_design* d, const double* g_rho, double* g_x, void* stream) {
  if (!d || !g_rho || !g_x) return PC_EINVAL;
  cudaGetLastError();
  cudaStream_t s = (cudaStream_t)stream;
  double* gphi = d->octant ? d->gphi : g_x;
  k_project_grad<<<cdiv(d->nnodes, 256), 256, 0, s>>>(g_rho, d->dmu, d->table, d->class_start, d->nclass, d->n[1],
                                                       d->n[2], d->nd[0], d->nd[1], d->nd[2], d->spacing, gphi);
  PC_LAUNCH_CHECK();
  if (d->octant) {
    k_octant_fold<<<cdiv(d->nvars, 256), 256, 0, s>>>(gphi, d->nd[0], d->nd[1], d->nd[2], g_x);
    PC_LAUNCH_CHECK();
  }
  return PC_OK;
}

extern "C" void pc_design_destroy(pc_design* d) {
  if (!d) return;
  if (d->table) cudaFree(d->table);
  if (d->class_start) cudaFree(d->class_start);
  if (d->phi) cudaFree(d->phi);
  if (d->gphi) cudaFree(d->gphi);
  if (d->dmu) cudaFree(d->dmu);
  delete d;
}
