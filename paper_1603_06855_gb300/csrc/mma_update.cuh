// One design variable's step of the method of moving asymptotes (Svanberg, Int. J. Numer. Meth.
// Eng. 24, 1987; asymptote and move-limit rules of his 2007 course notes) for the design problem
// of eq. topopt, which bounds the densities and has no other constraint, so every variable's
// convex subproblem is solved in closed form.  Host and device: the same function runs in
// k_mma_step and in a host build used to check it.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define PC_HD __host__ __device__ __forceinline__
#else
#define PC_HD inline
#endif

// x: current value; df: d(objective)/dx of the objective being MAXIMISED.
// xo1, xo2: the two previous values; low, upp: the previous asymptotes (all four ignored for
// iter < 2).  On return they hold the values for the next call, and *xnew the new value.
PC_HD void mma_box_update(double x, double df, int iter, double xmin, double xmax, double* xo1, double* xo2,
                          double* low, double* upp, double* xnew) {
  const double span = xmax - xmin;
  double L, U;
  if (iter < 2) {
    L = x - 0.5 * span;
    U = x + 0.5 * span;
  } else {
    // Shrink the asymptote distances where x oscillates, widen them where it keeps its direction.
    const double trend = (x - *xo1) * (*xo1 - *xo2);
    const double g = trend < 0.0 ? 0.7 : (trend > 0.0 ? 1.2 : 1.0);
    L = x - g * (*xo1 - *low);
    U = x + g * (*upp - *xo1);
    L = fmin(fmax(L, x - 10.0 * span), x - 0.01 * span);
    U = fmin(fmax(U, x + 0.01 * span), x + 10.0 * span);
  }
  const double alpha = fmax(fmax(xmin, L + 0.1 * (x - L)), x - 0.5 * span);
  const double beta = fmin(fmin(xmax, U - 0.1 * (U - x)), x + 0.5 * span);
  // Minimise g = -f through the model p / (U - x) + q / (x - L), whose slope at x is dg.
  const double dg = -df;
  const double pos = fmax(dg, 0.0), neg = fmax(-dg, 0.0), reg = 1e-5 / span;
  const double p = (U - x) * (U - x) * (1.001 * pos + 0.001 * neg + reg);
  const double q = (x - L) * (x - L) * (0.001 * pos + 1.001 * neg + reg);
  const double sp = sqrt(p), sq = sqrt(q);
  const double xs = (sp * L + sq * U) / (sp + sq);
  *xnew = fmin(fmax(xs, alpha), beta);
  *xo2 = *xo1;
  *xo1 = x;
  *low = L;
  *upp = U;
}
