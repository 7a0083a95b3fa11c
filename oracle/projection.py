"""Design parametrisation of the optimization (oracle; test infrastructure): reduced design field,
Heaviside projection and the SC mirror symmetry, with their chain rule.

Methods, "Topology optimization formulation" (the passage after eq. ``sensitivityew``): the
element densities rho_e are a closed-form function of an independent design field whose
variables are spaced at twice the element size (a reduced design variable field), through the
Heaviside Projection Method with a continuation on beta starting at beta = 1.  Results,
"Topology optimized structures": the SC runs optimise one eighth of the cell and generate the
rest by reflection.

Readings (the paper leaves the details to the cited HPM work):

* design nodes sit at the centres of the 2 x 2 x 2 element blocks, fractional position
  (2a + 1) / n per axis (spacing 2); spacing 1 puts one node at every element centroid;
* element e averages the node values phi_a within the projection radius r with the linear
  weights w_ea = r - |x_a - x_e| (Cartesian distance, nearest periodic image):
  mu_e = sum_a w_ea phi_a / sum_a w_ea;
* Heaviside projection for a minimum length scale of the rho = 1 phase:
  rho_e = 1 - exp(-beta mu_e) + mu_e exp(-beta), so rho(0) = 0, rho(1) = 1, rho -> mu as
  beta -> 0 and rho -> (mu > 0) as beta -> infinity;
* the printed radius, 1.4 % of the cell, lies below the distance from an element centroid to
  the nearest design node on the paper's own meshes (24^3 and 48^3), so it is read as 1.4
  element edge lengths; the radius is a parameter here;
* SC mirror symmetry: the free variables are the design nodes of one octant (n_d / 2 per axis,
  n_d even) and the full design grid is their image under the reflections a -> n_d - 1 - a
  (x -> -x about the lattice point, which maps the node grid onto itself).

Everything is built from dense pairwise distances, for small grids.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import lattice as lat


def heaviside(mu, beta: float):
    return 1.0 - np.exp(-beta * mu) + mu * np.exp(-beta)


def dheaviside(mu, beta: float):
    return beta * np.exp(-beta * mu) + np.exp(-beta)


def design_grid(n, spacing: int):
    """Design-grid shape and fractional node positions (nd, 3), C order."""
    n = tuple(int(v) for v in n)
    if spacing not in (1, 2) or any(v % spacing for v in n):
        raise ValueError("spacing must be 1 or 2 and divide every grid dimension")
    nd = tuple(v // spacing for v in n)
    idx = np.indices(nd).reshape(3, -1).T.astype(float)
    pos = (spacing * idx + spacing / 2.0) / np.array(n, float)
    return nd, pos


def filter_matrix(lattice: str, n, spacing: int, radius: float, a: float = 1.0) -> np.ndarray:
    """F (ne x nnodes): mu = F phi, each row the normalised linear weights of the nodes within
    radius (nearest periodic image among the 27 neighbouring cells)."""
    A = lat.primitive_vectors(lattice, a)
    s_e = lat.voxel_centroids(n)
    nd, s_a = design_grid(n, spacing)
    diff = s_a[None, :, :] - s_e[:, None, :]
    dist = np.full(diff.shape[:2], np.inf)
    for sh in itertools.product((-1, 0, 1), repeat=3):
        d = np.linalg.norm((diff + np.array(sh, float)) @ A.T, axis=2)
        dist = np.minimum(dist, d)
    W = np.maximum(radius - dist, 0.0)
    tot = W.sum(axis=1)
    if np.any(tot <= 0.0):
        raise ValueError("an element has no design node within the projection radius")
    return W / tot[:, None]


def octant_index(nd) -> np.ndarray:
    """For every node of the full design grid, the flat index of its octant image."""
    if any(v % 2 for v in nd):
        raise ValueError("the octant needs an even design grid")
    h = tuple(v // 2 for v in nd)
    f = [np.minimum(np.arange(v), v - 1 - np.arange(v)) for v in nd]
    i, j, l = np.meshgrid(f[0], f[1], f[2], indexing="ij")
    return ((i * h[1] + j) * h[2] + l).ravel()


def mirror_expand(x_oct: np.ndarray, nd) -> np.ndarray:
    return np.asarray(x_oct, float).ravel()[octant_index(nd)]


def mirror_fold(g_full: np.ndarray, nd) -> np.ndarray:
    """Adjoint of mirror_expand: every octant variable collects the gradient of its 8 images."""
    h = tuple(v // 2 for v in nd)
    out = np.zeros(h[0] * h[1] * h[2])
    np.add.at(out, octant_index(nd), np.asarray(g_full, float).ravel())
    return out


class DesignMap:
    """x (free variables) -> rho (element densities) and the chain rule back."""

    def __init__(self, lattice: str, n, spacing: int = 2, radius: float | None = None, octant: bool = False,
                 a: float = 1.0):
        A = lat.primitive_vectors(lattice, a)
        if radius is None:   # 1.4 element edge lengths (see the readings above)
            radius = 1.4 * np.linalg.norm(A[:, 0]) / n[0]
        if octant and lattice != "sc":
            raise ValueError("the mirror symmetry is the SC cell's")
        self.n = tuple(int(v) for v in n)
        self.nd, _ = design_grid(self.n, spacing)
        self.F = filter_matrix(lattice, self.n, spacing, radius, a)
        self.octant = octant

    @property
    def nvars(self) -> int:
        nd = int(np.prod(self.nd))
        return nd // 8 if self.octant else nd

    def phi(self, x):
        return mirror_expand(x, self.nd) if self.octant else np.asarray(x, float).ravel()

    def mu(self, x) -> np.ndarray:
        """The filtered field; a convex combination of values in [0, 1], clamped to [0, 1] only to
        remove rounding excursions."""
        return np.clip(self.F @ self.phi(x), 0.0, 1.0)

    def forward(self, x, beta: float) -> np.ndarray:
        return heaviside(self.mu(x), beta).reshape(self.n)

    def backward(self, x, beta: float, g_rho) -> np.ndarray:
        """dG/dx from dG/drho (chain rule through projection, filter and mirror)."""
        mu = self.mu(x)
        g_phi = self.F.T @ (np.asarray(g_rho, float).ravel() * dheaviside(mu, beta))
        return mirror_fold(g_phi, self.nd) if self.octant else g_phi
