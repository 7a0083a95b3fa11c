"""Cubic primitive cells, reciprocal basis and the plane-wave index set (oracle; test infrastructure).

Methods, "Study of cubic unit cells": band structures are computed on the
primitive cells of SC, BCC and FCC lattices, whose vectors run along the cube
edges, body diagonals and face diagonals.  Results, test functions after eq.
``mixedvariation``: f = exp[i 2 pi K.x] with K = T_1 (Q_1 + alpha) + T_2 (Q_2 + beta)
+ T_3 (Q_3 + gamma), Q the wavevector in reciprocal-lattice coordinates and T the
reciprocal basis (no factor 2 pi, so b_i . a_j = delta_ij).
"""
from __future__ import annotations

import numpy as np


def primitive_vectors(lattice: str, a: float = 1.0) -> np.ndarray:
    """Columns a_1, a_2, a_3 of the primitive cell, in the units of ``a``."""
    if lattice == "sc":
        A = np.eye(3)
    elif lattice == "bcc":
        A = 0.5 * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]]).T
    elif lattice == "fcc":
        A = 0.5 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]]).T
    else:
        raise ValueError(lattice)
    return a * A


def reciprocal_basis(A: np.ndarray) -> np.ndarray:
    """T with columns b_i such that b_i . a_j = delta_ij (the paper's T, no 2 pi)."""
    return np.linalg.inv(A).T


def cell_volume(A: np.ndarray) -> float:
    return abs(float(np.linalg.det(A)))


def plane_wave_indices(M: int) -> np.ndarray:
    """(alpha, beta, gamma) in [-M, M]^3, alpha slowest, gamma fastest: shape ((2M+1)^3, 3)."""
    r = np.arange(-M, M + 1)
    a, b, c = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)


def wavevectors(T: np.ndarray, Q, g: np.ndarray) -> np.ndarray:
    """K_p = T (Q + g_p), Cartesian, shape (N, 3)."""
    return (np.asarray(Q, float)[None, :] + g) @ T.T


def voxel_centroids(n) -> np.ndarray:
    """Element centroids in fractional coordinates s = ((i+1/2)/n0, (j+1/2)/n1, (l+1/2)/n2),
    C order (i slowest): shape (n0 n1 n2, 3)."""
    axes = [(np.arange(k) + 0.5) / k for k in n]
    i, j, l = np.meshgrid(*axes, indexing="ij")
    return np.stack([i.ravel(), j.ravel(), l.ravel()], axis=1)
