"""Dense FP64 assembly and solve of the mixed-variational band problem (oracle; test infrastructure).

Follows the paper step by step:

1. Material fields per element (Methods, eq. ``combinematerial`` and the linear
   element derivatives of eqs. ``diffOmega`` / ``diffPhi``): mass density and the
   isotropic compliance tensor are interpolated linearly between the two phases in
   chi_e = rho_e^p (p = 1 is the paper's linear law; rho_e = 1 is ``phase1``).
2. Element-sum quadrature (Methods, eqs. ``loop`` and ``matrixofintegral``): every
   integral of eqs. ``intH``, ``intOmega``, ``intPhi`` is the sum over elements of the
   integrand at the element centroid times the element volume, i.e. the matrix
   I = F^H diag(c_e v_e) F with F[e, q] = exp(i 2 pi K_q . x_e); the wavevector Q
   cancels in K_q - K_p, so every matrix is k-independent.
3. Omega (3N x 3N): the density integral on each displacement component; Phi
   (6N x 6N): the compliance integral on the six Voigt stress components (order 11,
   22, 33, 23, 13, 12 with engineering shear); H (3N x 6N): i 2 pi K^(row) times the
   plain element sum, contracted with the strain-transpose pattern E(K).
4. The condensed pencil of eq. ``matrixform``, H Phi^-1 H^H U = lambda Omega U, with
   ``*`` read as the conjugate transpose, solved by Cholesky solves and LAPACK's
   generalized Hermitian eigensolver; theta^H Omega theta = 1 and the eliminated
   stress coefficients are s = Phi^-1 H^H theta.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import lattice as lat

TWO_PI = 2.0 * np.pi


def compliance_voigt(E: float, nu: float) -> np.ndarray:
    """Isotropic compliance in Voigt form: stress (11,22,33,23,13,12) -> engineering strain."""
    D = np.zeros((6, 6))
    D[:3, :3] = -nu / E
    D[np.arange(3), np.arange(3)] = 1.0 / E
    D[np.arange(3, 6), np.arange(3, 6)] = 2.0 * (1.0 + nu) / E
    return D


def strain_transpose(K: np.ndarray) -> np.ndarray:
    """E(K), 3 x 6: row c, column v such that the engineering strain of a plane wave
    U exp(i 2 pi K.x) is i 2 pi E(K)^T U."""
    k1, k2, k3 = K
    return np.array([[k1, 0, 0, 0, k3, k2],
                     [0, k2, 0, k3, 0, k1],
                     [0, 0, k3, k2, k1, 0]], dtype=float)


@dataclasses.dataclass
class Problem:
    lattice: str
    a: float
    n: tuple
    M: int
    A: np.ndarray
    T: np.ndarray
    V: float
    g: np.ndarray
    s: np.ndarray
    x: np.ndarray
    ve: float
    chi: np.ndarray
    dchi: np.ndarray
    rho_m: np.ndarray
    D: np.ndarray
    d_rho: float
    d_D: np.ndarray       # dD/dchi: (6, 6), or (ne, 6, 6) under the Young's-modulus law
    F: np.ndarray
    I: np.ndarray
    Omega: np.ndarray
    Phi: np.ndarray
    _phi_cho: object = None
    _phi_inv: np.ndarray | None = None

    @property
    def N(self) -> int:
        return self.g.shape[0]

    def phi_cho(self):
        if self._phi_cho is None:
            self._phi_cho = sla.cho_factor(self.Phi, lower=True)
        return self._phi_cho

    def phi_inv(self) -> np.ndarray:
        if self._phi_inv is None:
            self._phi_inv = sla.cho_solve(self.phi_cho(), np.eye(self.Phi.shape[0], dtype=complex))
        return self._phi_inv


def material_fields(rho: np.ndarray, phase1: dict, phase0: dict, penal: float, law: str = "compliance"):
    """chi = rho^p, dchi/drho, interpolated density and compliance per element, and dD/dchi.

    law "compliance": density and compliance linear in chi, so dD/dchi is the constant
    difference of the phases (the element derivatives of eqs. diffOmega / diffPhi).
    law "young": eq. combinematerial read literally, Young's modulus linear in chi (and
    Poisson's ratio with it); each element has the compliance of its interpolated isotropic
    material, D = (1/E) P1 + (nu/E) P2 with P1 = diag(1,1,1,2,2,2) and P2 = 2 on the shear
    diagonal, -1 between normal components, so dD/dchi varies per element: (ne, 6, 6)."""
    r = np.asarray(rho, float).ravel()
    chi = r ** penal
    dchi = penal * r ** (penal - 1.0) if penal != 1.0 else np.ones_like(r)
    rho_m = phase0["rho"] + chi * (phase1["rho"] - phase0["rho"])
    if law == "compliance":
        D1 = compliance_voigt(phase1["E"], phase1["nu"])
        D0 = compliance_voigt(phase0["E"], phase0["nu"])
        D = D0[None] + chi[:, None, None] * (D1 - D0)[None]
        return chi, dchi, rho_m, D, phase1["rho"] - phase0["rho"], D1 - D0
    if law != "young":
        raise ValueError(law)
    dE, dnu = phase1["E"] - phase0["E"], phase1["nu"] - phase0["nu"]
    E = phase0["E"] + chi * dE
    nu = phase0["nu"] + chi * dnu
    D = np.stack([compliance_voigt(e, v) for e, v in zip(E, nu)])
    P1 = np.diag([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])
    P2 = np.zeros((6, 6))
    P2[:3, :3] = -1.0
    P2[np.arange(3), np.arange(3)] = 0.0
    P2[np.arange(3, 6), np.arange(3, 6)] = 2.0
    da = -dE / E ** 2                      # d(1/E)/dchi
    db = (dnu * E - nu * dE) / E ** 2      # d(nu/E)/dchi
    d_D = da[:, None, None] * P1[None] + db[:, None, None] * P2[None]
    return chi, dchi, rho_m, D, phase1["rho"] - phase0["rho"], d_D


def element_sum(F: np.ndarray, w: np.ndarray) -> np.ndarray:
    """I_pq = sum_e w_e conj(F[e,p]) F[e,q] (the outer-product form of eq. ``matrixofintegral``)."""
    return (F.conj().T * w[None, :]) @ F


def build(lattice: str, n, M: int, rho, phase1: dict, phase0: dict, penal: float = 1.0,
          a: float = 1.0, law: str = "compliance") -> Problem:
    A = lat.primitive_vectors(lattice, a)
    T = lat.reciprocal_basis(A)
    V = lat.cell_volume(A)
    g = lat.plane_wave_indices(M)
    s = lat.voxel_centroids(n)
    x = s @ A.T
    ne = s.shape[0]
    ve = V / ne
    chi, dchi, rho_m, D, d_rho, d_D = material_fields(rho, phase1, phase0, penal, law)
    K0 = g @ T.T  # Q-independent part of K_q
    F = np.exp(1j * TWO_PI * (x @ K0.T))
    N = g.shape[0]
    I = element_sum(F, np.full(ne, ve))
    Tr = element_sum(F, rho_m * ve)
    Omega = np.kron(np.eye(3), Tr)
    # Phi[(v,p),(w,q)] = sum_e D_e[v,w] v_e conj(F[e,p]) F[e,q]; equal fields are summed once.
    Phi = np.zeros((6 * N, 6 * N), dtype=complex)
    cache = {}
    for v in range(6):
        for w in range(6):
            field = D[:, v, w]
            if not np.any(field):
                continue
            key = field.tobytes()
            if key not in cache:
                cache[key] = element_sum(F, field * ve)
            Phi[v * N:(v + 1) * N, w * N:(w + 1) * N] = cache[key]
    return Problem(lattice, a, tuple(n), M, A, T, V, g, s, x, ve, chi, dchi, rho_m, D, d_rho, d_D,
                   F, I, Omega, Phi)


def from_workload(w) -> Problem:
    return build(w.lattice, w.n, w.M, w.rho, w.phase1, w.phase0, w.penal, w.a)


def coupling(P: Problem, Q, literal: bool = True) -> np.ndarray:
    """H (3N x 6N) of eq. ``intH``: H[(c,p),(v,q)] = i 2 pi E(K_p)[c,v] I_pq.

    ``literal=False`` keeps only the diagonal p = q, where the centroid sum of a
    non-zero plane-wave difference vanishes whenever every n_i >= 2M+1."""
    N = P.N
    K = lat.wavevectors(P.T, Q, P.g)
    E = np.stack([strain_transpose(k) for k in K])  # (N,3,6)
    H = np.zeros((3 * N, 6 * N), dtype=complex)
    Iuse = P.I if literal else np.diag(np.diag(P.I))
    for c in range(3):
        for v in range(6):
            H[c * N:(c + 1) * N, v * N:(v + 1) * N] = 1j * TWO_PI * E[:, c, v][:, None] * Iuse
    return H


def operator(P: Problem, Q, literal: bool | None = None) -> tuple[np.ndarray, np.ndarray]:
    """A = H Phi^-1 H^H (eq. ``matrixform``) and H."""
    if literal is None:
        literal = P.N <= 343
    H = coupling(P, Q, literal)
    if literal:
        Z = sla.cho_solve(P.phi_cho(), H.conj().T)
        A = H @ Z
    else:
        # H is block diagonal in the plane-wave index: contract blockwise with Phi^-1.
        N = P.N
        Hb = np.stack([H[c * N:(c + 1) * N, :].reshape(N, 6, N)[np.arange(N), :, np.arange(N)]
                       for c in range(3)], axis=1)  # (N, 3, 6): H[(c,p),(v,p)]
        Pinv = P.phi_inv().reshape(6, N, 6, N)
        X = np.einsum("pcv,vpwq->cpwq", Hb, Pinv, optimize=True)
        A = np.einsum("cpwq,qdw->cpdq", X, Hb.conj(), optimize=True).reshape(3 * N, 3 * N)
    A = 0.5 * (A + A.conj().T)
    return A, H


@dataclasses.dataclass
class KSolution:
    lam: np.ndarray     # (nb,) ascending
    theta: np.ndarray   # (3N, nb), theta^H Omega theta = 1
    s: np.ndarray       # (6N, nb) stress coefficients Phi^-1 H^H theta


def solve_k(P: Problem, Q, nb: int, literal: bool | None = None) -> KSolution:
    A, H = operator(P, Q, literal)
    lam, theta = sla.eigh(A, P.Omega, subset_by_index=[0, nb - 1])
    s = sla.cho_solve(P.phi_cho(), H.conj().T @ theta)
    return KSolution(lam, theta, s)


def bands(P: Problem, Qs, nb: int, literal: bool | None = None, keep: bool = False):
    """Lowest nb eigenvalues lambda = omega^2 at every wavevector: (nk, nb); optionally the solutions."""
    sols = [solve_k(P, Q, nb, literal) for Q in np.asarray(Qs, float)]
    lam = np.array([s.lam for s in sols])
    return (lam, sols) if keep else lam


def omega(lam: np.ndarray) -> np.ndarray:
    return np.sqrt(np.maximum(lam, 0.0))
