"""Eigenvalue sensitivities d lambda / d rho_e (oracle; test infrastructure).

Methods, eqs. ``normalev`` and ``sensitivityew``: with left and right eigenvectors
psi, theta normalised by psi^* theta = 1,

    d lambda / d rho_e = psi^* [ -Omega^-1 dOmega Omega^-1 (H Phi^-1 H^*)
                                 - Omega^-1 (H Phi^-1 dPhi Phi^-1 H^*) ] theta,

and eqs. ``diffOmega`` / ``diffPhi`` give the per-element derivative matrices
dOmega/drho_e = (rho^1 - rho^2) f^(e)_pq v^(e), dPhi/drho_e = (D^1 - D^2) f^(e)_pq v^(e)
(times d chi / d rho under the power law).  The pencil is Hermitian with Omega
positive definite, so psi = Omega theta and the expression equals

    d lambda / d rho_e = -lambda theta^H dOmega theta - s^H dPhi s,   s = Phi^-1 H^H theta,

which, since f^(e)_pq = conj(F[e,p]) F[e,q], is a pair of quadratic forms of the
displacement and stress fields synthesised at the element centroid:

    chi'_e v_e [ -lambda (rho^1 - rho^0) sum_c |u_c(x_e)|^2 - sigma(x_e)^H (D^1 - D^0) sigma(x_e) ].

``literal`` builds the per-element matrices and evaluates the first form (tiny
cases); ``voxel`` evaluates the last.
"""
from __future__ import annotations

import numpy as np

from . import mixed


def voxel(P: mixed.Problem, lam: float, theta: np.ndarray, s: np.ndarray) -> np.ndarray:
    """d lambda / d rho_e for every element from one eigenpair (theta: 3N, s: 6N)."""
    N = P.N
    u = P.F @ theta.reshape(3, N).T        # (ne, 3) displacement at centroids
    sig = P.F @ s.reshape(6, N).T          # (ne, 6) Voigt stress at centroids
    mass = np.sum(np.abs(u) ** 2, axis=1)
    sub = "ev,vw,ew->e" if P.d_D.ndim == 2 else "ev,evw,ew->e"   # per-element dD/dchi (Young's-modulus law)
    comp = np.real(np.einsum(sub, sig.conj(), P.d_D, sig))
    return P.dchi * P.ve * (-lam * P.d_rho * mass - comp)


def literal(P: mixed.Problem, Q, lam: float, theta: np.ndarray) -> np.ndarray:
    """Eq. ``sensitivityew`` with explicit per-element matrices (cost ~ ne * (6N)^2; tiny only)."""
    N = P.N
    A, H = mixed.operator(P, Q, literal=True)
    Oinv = np.linalg.inv(P.Omega)
    Phinv = np.linalg.inv(P.Phi)
    psi = P.Omega @ theta
    HPH = H @ Phinv @ H.conj().T
    out = np.zeros(P.F.shape[0])
    for e in range(P.F.shape[0]):
        f = np.outer(P.F[e].conj(), P.F[e]) * P.ve          # f^(e)_pq v^(e)
        dOm = P.dchi[e] * np.kron(np.eye(3), P.d_rho * f)
        dPh = P.dchi[e] * np.kron(P.d_D if P.d_D.ndim == 2 else P.d_D[e], f)
        term = (-Oinv @ dOm @ Oinv @ HPH - Oinv @ (H @ Phinv @ dPh @ Phinv @ H.conj().T))
        out[e] = np.real(psi.conj() @ term @ theta)
    return out


def weighted(P: mixed.Problem, sols, weights: np.ndarray) -> np.ndarray:
    """sum_{k,b} w[k,b] d lambda_{k,b} / d rho_e over the (k, b) with non-zero weight."""
    g = np.zeros(P.F.shape[0])
    for k, sol in enumerate(sols):
        for b in np.nonzero(weights[k])[0]:
            g += weights[k, b] * voxel(P, sol.lam[b], sol.theta[:, b], sol.s[:, b])
    return g
