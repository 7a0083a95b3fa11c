// Design update of the optimization loop (Methods, eq. topopt: maximise the gap with
// 0 <= rho_e <= 1): one step of the method of moving asymptotes on every design variable.
// Elementwise and HBM bound: each variable reads and writes its value, its two previous
// values and its two asymptotes, and reads its gradient (88 bytes).
#include <cmath>

#include "kernels.h"
#include "mma_update.cuh"

__global__ __launch_bounds__(256) void k_mma_step(long long n, double* __restrict__ x, const double* __restrict__ df,
                                                  double* __restrict__ xo1, double* __restrict__ xo2,
                                                  double* __restrict__ low, double* __restrict__ upp, int iter,
                                                  double xmin, double xmax) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = xo1[i], b = xo2[i], L = low[i], U = upp[i], xn;
  mma_box_update(x[i], df[i], iter, xmin, xmax, &a, &b, &L, &U, &xn);
  x[i] = xn;
  xo1[i] = a;
  xo2[i] = b;
  low[i] = L;
  upp[i] = U;
}

extern "C" int pc_mma_step(long long n, double* x_dev, const double* df_dev, double* xold1_dev, double* xold2_dev,
                           double* low_dev, double* upp_dev, int iter, double xmin, double xmax, void* stream) {
  if (n < 1 || !x_dev || !df_dev || !xold1_dev || !xold2_dev || !low_dev || !upp_dev || iter < 0) return PC_EINVAL;
  if (!std::isfinite(xmin) || !std::isfinite(xmax) || !(xmax > xmin)) return PC_EINVAL;
  if ((n + 255) / 256 > 0x7fffffffLL) return PC_EINVAL;
  cudaGetLastError();  // the launch check below reports only this launch
  k_mma_step<<<cdiv(n, 256), 256, 0, (cudaStream_t)stream>>>(n, x_dev, df_dev, xold1_dev, xold2_dev, low_dev,
                                                                upp_dev, iter, xmin, xmax);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
