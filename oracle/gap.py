"""Normalized band gap between bands n and n+1 and its gradient weights (oracle; test infrastructure).

Methods, eq. ``obj``: f = 2 (min_k lambda_{t+1} - max_k lambda_t) / (min_k lambda_{t+1}
+ max_k lambda_t).  Results, "A note on normalized band gaps": the reported quantity
is gap width over mid-gap frequency, i.e. the same formula in omega = sqrt(lambda);
every gap percentage the paper prints follows the omega form, which is the default.

The max / min are not smooth; the gradient flows through the extremal (k, band)
only.  Exact ties in k are broken by the lowest k index.  Bands at the extremal k
whose eigenvalue lies within ``rel_tol`` of the extremal one form a degenerate
cluster, and each member receives an equal share of the weight: that is the
gradient of the cluster-mean eigenvalue, independent of the basis chosen inside
the cluster.
"""
from __future__ import annotations

import dataclasses

import numpy as np

MODE_OMEGA = 0
MODE_LAMBDA = 1


@dataclasses.dataclass
class GapResult:
    gap: float
    lower: float   # a = max_k band n (omega or lambda)
    upper: float   # b = min_k band n+1
    k_lower: int
    k_upper: int
    weights: np.ndarray  # (nk, nb): dG/dlambda_{k,b}


def gap(lam: np.ndarray, n_lower: int, mode: int = MODE_OMEGA, rel_tol: float = 1e-8) -> GapResult:
    """Gap between 1-based band ``n_lower`` and ``n_lower + 1`` of a band table lam (nk, nb)."""
    lam = np.asarray(lam, float)
    nk, nb = lam.shape
    if not (1 <= n_lower < nb):
        raise ValueError("n_lower out of range")
    lo = lam[:, n_lower - 1]
    hi = lam[:, n_lower]
    k_a = int(np.argmax(lo))   # first occurrence: lowest k among ties
    k_b = int(np.argmin(hi))
    la, lb = lo[k_a], hi[k_b]
    w = np.zeros_like(lam)
    if mode == MODE_OMEGA:
        a, b = np.sqrt(max(la, 0.0)), np.sqrt(max(lb, 0.0))
        G = 2.0 * (b - a) / (b + a)
        # dG/da = -4b/(a+b)^2, dG/db = 4a/(a+b)^2, d omega / d lambda = 1 / (2 omega)
        wa = -2.0 * b / (a * (a + b) ** 2) if a > 0 else 0.0
        wb = 2.0 * a / (b * (a + b) ** 2) if b > 0 else 0.0
    elif mode == MODE_LAMBDA:
        a, b = la, lb
        G = 2.0 * (b - a) / (b + a)
        wa = -4.0 * b / (a + b) ** 2
        wb = 4.0 * a / (a + b) ** 2
    else:
        raise ValueError(mode)
    for k, band, wt in ((k_a, n_lower - 1, wa), (k_b, n_lower, wb)):
        ref = lam[k, band]
        cluster = np.nonzero(np.abs(lam[k] - ref) <= rel_tol * abs(ref))[0]
        w[k, cluster] += wt / len(cluster)
    return GapResult(float(G), float(a), float(b), k_a, k_b, w)


def ks_gap(lam: np.ndarray, n_lower: int, beta: float, omega_ref: float, rel_tol: float = 1e-8) -> GapResult:
    """Smooth (Kreisselmeier-Steinhauser) surrogate of the omega-form gap.

    Not in the paper: its objective takes the max over k of band n and the min of band n + 1,
    which is not differentiable where the extremal k changes.  Here, with x = omega / omega_ref,
        a = omega_ref (1/beta) log sum_k exp(beta x_{k,n}),   b = -omega_ref (1/beta) log sum_k exp(-beta x_{k,n+1}),
    G = 2 (b - a) / (b + a).  a >= max_k omega_n and b <= min_k omega_{n+1}, so G is below the
    exact gap and tends to it as beta grows.  omega_ref is a fixed scale (not a function of the
    bands), so a and b are smooth.  dG/dlambda_{k,b} follows by the chain rule with
    d omega / d lambda = 1 / (2 omega); at each k the weight of band n (and of band n + 1) is
    shared equally by the bands within rel_tol of it, as in gap()."""
    lam = np.asarray(lam, float)
    nk, nb = lam.shape
    if not (1 <= n_lower < nb):
        raise ValueError("n_lower out of range")
    lo, hi = n_lower - 1, n_lower
    x = np.sqrt(np.maximum(lam[:, lo], 0.0)) / omega_ref
    y = np.sqrt(np.maximum(lam[:, hi], 0.0)) / omega_ref
    xm, ym = x.max(), y.min()
    ea = np.exp(beta * (x - xm))
    eb = np.exp(-beta * (y - ym))
    a = xm + np.log(ea.sum()) / beta
    b = ym - np.log(eb.sum()) / beta
    G = 2.0 * (b - a) / (b + a)
    dGda = -4.0 * b / (a + b) ** 2
    dGdb = 4.0 * a / (a + b) ** 2
    p, q = ea / ea.sum(), eb / eb.sum()
    w = np.zeros_like(lam)
    lref = omega_ref ** 2
    for k in range(nk):
        for band, xv, wt in ((lo, x[k], dGda * p[k]), (hi, y[k], dGdb * q[k])):
            if xv <= 0.0:
                continue
            wl = wt / (2.0 * xv * lref)   # d x / d lambda = 1 / (2 x omega_ref^2)
            ref = lam[k, band]
            cluster = np.nonzero(np.abs(lam[k] - ref) <= rel_tol * abs(ref))[0]
            w[k, cluster] += wl / len(cluster)
    return GapResult(float(G), float(a * omega_ref), float(b * omega_ref), int(np.argmax(x)), int(np.argmin(y)), w)
