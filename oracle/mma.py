"""One step of the method of moving asymptotes for the box-constrained design problem
(oracle; test infrastructure).

Methods, eq. ``topopt``: maximise the gap f(rho) subject to the eigenproblem and
0 <= rho_e <= 1 only (no volume constraint).  The paper names no optimizer; this is
Svanberg's method of moving asymptotes (Int. J. Numer. Meth. Eng. 24, 1987; the
asymptote and move-limit rules of his 2007 course notes), written for a problem with
no constraints besides the bounds, where it needs no dual solve:

* the objective to minimise is g = -f with gradient dg = -df;
* asymptotes L < x < U: at the first two iterations x -/+ 0.5 (xmax - xmin); later
  the previous distances scaled by 0.7 where x oscillated (the last two moves of
  opposite sign), 1.2 where it moved twice the same way, 1 otherwise, kept within
  [0.01, 10] (xmax - xmin) of x;
* move limits alpha = max(xmin, L + 0.1 (x - L), x - 0.5 (xmax - xmin)) and
  beta = min(xmax, U - 0.1 (U - x), x + 0.5 (xmax - xmin));
* the convex separable model g(x) ~ sum_j p_j / (U_j - x_j) + q_j / (x_j - L_j) + const with
  p = (U - x)^2 (1.001 max(dg, 0) + 0.001 max(-dg, 0) + 1e-5 / (xmax - xmin)),
  q = (x - L)^2 (0.001 max(dg, 0) + 1.001 max(-dg, 0) + 1e-5 / (xmax - xmin));
* each term is convex on (L, U) with its minimum where p / (U - x)^2 = q / (x - L)^2,
  x* = (sqrt(p) L + sqrt(q) U) / (sqrt(p) + sqrt(q)), clipped to [alpha, beta].
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class MMAState:
    """Iterates and asymptotes carried from step to step."""
    it: int = 0
    x1: np.ndarray | None = None   # previous iterate
    x2: np.ndarray | None = None   # the one before
    L: np.ndarray | None = None
    U: np.ndarray | None = None


def asymptotes(x, st: MMAState, xmin=0.0, xmax=1.0):
    span = xmax - xmin
    if st.it < 2:
        return x - 0.5 * span, x + 0.5 * span
    trend = (x - st.x1) * (st.x1 - st.x2)
    gamma = np.where(trend < 0, 0.7, np.where(trend > 0, 1.2, 1.0))
    L = x - gamma * (st.x1 - st.L)
    U = x + gamma * (st.U - st.x1)
    L = np.clip(L, x - 10.0 * span, x - 0.01 * span)
    U = np.clip(U, x + 0.01 * span, x + 10.0 * span)
    return L, U


def step(x, df, st: MMAState, xmin=0.0, xmax=1.0):
    """Ascent step on f: returns the next iterate and advances the state in place."""
    x = np.asarray(x, float)
    dg = -np.asarray(df, float)
    span = xmax - xmin
    L, U = asymptotes(x, st, xmin, xmax)
    alpha = np.maximum.reduce([np.full_like(x, xmin), L + 0.1 * (x - L), x - 0.5 * span])
    beta = np.minimum.reduce([np.full_like(x, xmax), U - 0.1 * (U - x), x + 0.5 * span])
    pos, neg = np.maximum(dg, 0.0), np.maximum(-dg, 0.0)
    p = (U - x) ** 2 * (1.001 * pos + 0.001 * neg + 1e-5 / span)
    q = (x - L) ** 2 * (0.001 * pos + 1.001 * neg + 1e-5 / span)
    sp, sq = np.sqrt(p), np.sqrt(q)
    xn = np.clip((sp * L + sq * U) / (sp + sq), alpha, beta)
    st.x2, st.x1 = st.x1, x.copy()
    st.L, st.U = L, U
    st.it += 1
    return xn
