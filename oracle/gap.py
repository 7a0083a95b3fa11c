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
