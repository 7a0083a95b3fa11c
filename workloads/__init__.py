"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

This module holds only input preparation: material constants, the workload
configurations, seeded density designs and Bloch wavevector paths.  It contains
none of the band-structure or sensitivity arithmetic, and it imports neither the
oracle nor the CUDA binding.

Workload recipe (the paper's optimized designs exist only as figures, so seeded
designs with the same shapes stand in for them):

* two-phase tungsten-carbide / epoxy cells on SC, BCC and FCC primitive cells,
  voxel densities rho_e in [0, 1] with rho_e = 1 the stiff, heavy phase;
* sc8_M1_binary_cube: SC 8^3 binary cube inclusion, M = 1, 10 k on G-X-M-G-R, 6 bands;
* sc16_M2_grf: SC 16^3 periodic Gaussian random field through a sigmoid, p = 3,
  M = 2, 30 k on the irreducible-zone boundary, 12 bands;
* bcc24_M3_grf: BCC 24^3 random field in fractional coordinates, M = 3, 64 k, 16 bands;
* fcc32_M4_levelset: FCC 32^3 smoothed level set of an 8-term trigonometric sum,
  M = 4 (729 plane waves), 100 k, 20 bands;
* batch32_mixed: 32 designs of mixed lattice, cutoff and grid, 48 k, 20 bands;
* sphere_inclusion: one sphere per primitive cell, as in the paper's volume-fraction scans.

Seeds: numpy.random.default_rng(SEED_BASE[workload] + design_index).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Material constants (SI).  phase1 is rho_e = 1, phase0 is rho_e = 0.
TUNGSTEN_CARBIDE = dict(rho=15800.0, E=600e9, nu=0.22)
EPOXY = dict(rho=1180.0, E=4.35e9, nu=0.37)
# The constants the paper quotes for its sphere scans (Results, normalized band gaps).
PAPER_WC = dict(rho=13800.0, E=387.5559e9, nu=0.3459)
PAPER_EPOXY = dict(rho=1180.0, E=4.3438e9, nu=0.3679)


# Primitive vectors (columns, units of the cubic lattice constant).  A private
# copy used only to express high-symmetry points in reduced coordinates.
def _primitive(lattice: str) -> np.ndarray:
    if lattice == "sc":
        return np.eye(3)
    if lattice == "bcc":
        return 0.5 * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]]).T
    if lattice == "fcc":
        return 0.5 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]]).T
    raise ValueError(lattice)


# High-symmetry points, Cartesian, units of 1/a (no 2*pi).
HIGH_SYMMETRY = {
    "sc": {"G": (0, 0, 0), "X": (0, 0.5, 0), "M": (0.5, 0.5, 0), "R": (0.5, 0.5, 0.5)},
    "bcc": {"G": (0, 0, 0), "H": (0, 0, 1), "N": (0.5, 0.5, 0), "P": (0.5, 0.5, 0.5)},
    "fcc": {"G": (0, 0, 0), "X": (0, 1, 0), "W": (0.5, 1, 0), "K": (0.75, 0.75, 0),
            "L": (0.5, 0.5, 0.5), "U": (0.25, 1, 0.25)},
}
# Boundary paths of the irreducible zones; '|' is a jump.
PATHS = {
    "sc": "G-X-M-G-R-X|M-R",
    "sc_short": "G-X-M-G-R",
    "bcc": "G-H-N-G-P-H|P-N",
    "fcc": "G-X-W-K-G-L-U-W-L-K|U-X",
}


def kpath(lattice: str, nk: int, path: str | None = None) -> np.ndarray:
    """nk wavevectors on a high-symmetry path, in reduced coordinates Q (nk, 3).

    Every vertex is included; the remaining points are shared between the
    segments in proportion to their length (largest remainder).  Q_j = K . a_j.
    """
    spec = PATHS[path or lattice]
    pts = HIGH_SYMMETRY[lattice]
    polylines = [[np.array(pts[s], float) for s in part.split("-")] for part in spec.split("|")]
    vertices = sum(len(p) for p in polylines)
    if nk < vertices:
        raise ValueError(f"need at least {vertices} points for path {spec}")
    segs = [(pl[i], pl[i + 1]) for pl in polylines for i in range(len(pl) - 1)]
    lens = np.array([np.linalg.norm(b - a) for a, b in segs])
    extra = nk - vertices
    share = extra * lens / lens.sum()
    alloc = np.floor(share).astype(int)
    order = np.argsort(-(share - alloc), kind="stable")
    alloc[order[: extra - alloc.sum()]] += 1
    out = []
    si = 0
    for pl in polylines:
        out.append(pl[0])
        for i in range(len(pl) - 1):
            a, b = pl[i], pl[i + 1]
            m = alloc[si]
            for t in range(1, m + 1):
                out.append(a + (b - a) * t / (m + 1))
            out.append(b)
            si += 1
    K = np.array(out)
    assert K.shape[0] == nk
    A = _primitive(lattice)
    return K @ A  # Q_j = K . a_j


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def gaussian_random_field(n: tuple[int, int, int], ell: float, rng, cart: np.ndarray | None = None):
    """Periodic Gaussian random field: white noise circularly filtered by exp(-|r|^2 / (2 ell^2)),
    standardised to zero mean and unit variance.  r is the minimum-image offset in fractional
    coordinates, mapped to Cartesian by ``cart`` when given."""
    w = rng.standard_normal(n)
    grids = np.meshgrid(*[np.arange(k) / k for k in n], indexing="ij")
    d = np.stack([(g + 0.5) % 1.0 - 0.5 for g in grids], axis=-1)
    if cart is not None:
        d = d @ cart.T
    kern = np.exp(-np.sum(d * d, axis=-1) / (2 * ell * ell))
    z = np.real(np.fft.ifftn(np.fft.fftn(w) * np.fft.fftn(kern)))
    z = (z - z.mean()) / z.std()
    return z


def trig_levelset_design(n: tuple[int, int, int], rng, terms: int = 8) -> np.ndarray:
    """Smooth single-network inclusion: phi(s) = sum_j a_j cos(2 pi m_j.s + phi_j),
    thresholded at its median and smoothed by a sigmoid of slope 8 / std(phi)."""
    ms = []
    while len(ms) < terms:
        m = rng.integers(-2, 3, size=3)
        if np.any(m != 0):
            ms.append(m)
    a = rng.standard_normal(terms)
    ph = rng.uniform(0.0, 2 * np.pi, size=terms)
    grids = np.meshgrid(*[(np.arange(k) + 0.5) / k for k in n], indexing="ij")
    s = np.stack(grids, axis=-1)
    phi = np.zeros(n)
    for j in range(terms):
        phi += a[j] * np.cos(2 * np.pi * (s @ ms[j]) + ph[j])
    t = np.median(phi)
    return _sigmoid(8.0 * (phi - t) / phi.std())


@dataclasses.dataclass
class Workload:
    """One design evaluation: lattice, grid, cutoff, bands, k-points, density."""
    name: str
    lattice: str
    n: tuple[int, int, int]
    M: int
    nbands: int
    Q: np.ndarray            # (nk, 3) reduced wavevectors
    rho: np.ndarray          # (n0, n1, n2) densities in [0, 1], C order
    penal: float
    gaps: tuple[int, ...]    # 1-based lower band of each requested gap
    seed: int
    a: float = 1.0
    phase1: dict = dataclasses.field(default_factory=lambda: dict(TUNGSTEN_CARBIDE))
    phase0: dict = dataclasses.field(default_factory=lambda: dict(EPOXY))

    @property
    def N(self) -> int:
        return (2 * self.M + 1) ** 3

    @property
    def nk(self) -> int:
        return self.Q.shape[0]


SEED_BASE = {"sc8_M1_binary_cube": 1603, "sc16_M2_grf": 2603, "bcc24_M3_grf": 3603,
             "fcc32_M4_levelset": 4603, "batch32_mixed": 5603}


def _seed(workload: str, design: int = 0) -> int:
    return SEED_BASE[workload] + design


def sc8_binary_cube() -> Workload:
    n = (8, 8, 8)
    rho = np.zeros(n)
    rho[2:6, 2:6, 2:6] = 1.0
    return Workload("sc8_M1_binary_cube", "sc", n, 1, 6, kpath("sc", 10, "sc_short"), rho,
                    1.0, (3,), _seed("sc8_M1_binary_cube"))


def sc16_grf(design: int = 0) -> Workload:
    seed = _seed("sc16_M2_grf", design)
    rng = np.random.default_rng(seed)
    n = (16, 16, 16)
    z = gaussian_random_field(n, 1.0 / 6.0, rng, cart=np.eye(3))
    return Workload("sc16_M2_grf", "sc", n, 2, 12, kpath("sc", 30), _sigmoid(z), 3.0, (3, 6), seed)


def bcc24_grf(design: int = 0) -> Workload:
    seed = _seed("bcc24_M3_grf", design)
    rng = np.random.default_rng(seed)
    n = (24, 24, 24)
    z = gaussian_random_field(n, 1.0 / 6.0, rng)
    return Workload("bcc24_M3_grf", "bcc", n, 3, 16, kpath("bcc", 64), _sigmoid(z), 3.0, (6,), seed)


def fcc32_levelset(design: int = 0) -> Workload:
    seed = _seed("fcc32_M4_levelset", design)
    rng = np.random.default_rng(seed)
    n = (32, 32, 32)
    rho = trig_levelset_design(n, rng)
    return Workload("fcc32_M4_levelset", "fcc", n, 4, 20, kpath("fcc", 100), rho, 3.0, (6,), seed)


def batch32_mixed() -> list[Workload]:
    """Uneven batch: 12 SC, 10 BCC, 10 FCC designs; N drawn from {125, 343, 729, 1331}."""
    out = []
    lattices = ["sc"] * 12 + ["bcc"] * 10 + ["fcc"] * 10
    for i, lat in enumerate(lattices):
        seed = _seed("batch32_mixed", i)
        rng = np.random.default_rng(seed)
        M = int(rng.choice([2, 3, 4, 5]))
        grid_choices = [g for g in (16, 20, 24, 28, 32, 36, 40) if g >= 2 * M + 1]
        g = int(rng.choice(grid_choices))
        n = (g, g, g)
        cart = np.eye(3) if lat == "sc" else None
        z = gaussian_random_field(n, 1.0 / 6.0, rng, cart=cart)
        out.append(Workload(f"{lat}{g}_M{M}_grf_{i}", lat, n, M, 20, kpath(lat, 48), _sigmoid(z),
                            3.0, (6,), seed))
    return out


WORKLOADS = {"sc8_M1_binary_cube": sc8_binary_cube, "sc16_M2_grf": sc16_grf,
             "bcc24_M3_grf": bcc24_grf, "fcc32_M4_levelset": fcc32_levelset}


def homogeneous(lattice: str, n, M: int, nbands: int, nk: int, value: float = 0.0) -> Workload:
    rho = np.full(tuple(n), float(value))
    return Workload(f"{lattice}_homog", lattice, tuple(n), M, nbands, kpath(lattice, nk), rho, 1.0, (3,), 0)


def laminate(n1: int, n_other: int, M: int, frac1: float, kx: list[float]) -> Workload:
    """SC cell layered along x: rho = 1 on the first round(frac1 * n1) voxel planes."""
    n = (n1, n_other, n_other)
    rho = np.zeros(n)
    rho[: int(round(frac1 * n1))] = 1.0
    Q = np.array([[k, 0.0, 0.0] for k in kx])
    return Workload("laminate", "sc", n, M, 6, Q, rho, 1.0, (1,), 0)


def random_design(n, rng, low=0.05, high=0.95) -> np.ndarray:
    return rng.uniform(low, high, size=tuple(n))


def high_symmetry_points(lattice: str) -> np.ndarray:
    """The distinct high-symmetry points of the irreducible zone, reduced coordinates (n, 3)."""
    A = _primitive(lattice)
    return np.array([np.array(p, float) @ A for p in HIGH_SYMMETRY[lattice].values()])


def sphere_inclusion(lattice: str, n, vf: float, sub: int = 3) -> np.ndarray:
    """One sphere per primitive cell, centred on the lattice points, of volume fraction vf.

    rho_e is the share of the voxel inside the sphere, estimated on sub^3 points per voxel
    (the voxel's own cell of a sub x sub x sub grid); the distance to the nearest lattice
    point uses the 27 neighbouring cells, which covers every point of the cell for these
    primitive vectors.  A = cubic lattice constant 1."""
    A = _primitive(lattice)
    V = abs(np.linalg.det(A))
    r = (3.0 * vf * V / (4.0 * math.pi)) ** (1.0 / 3.0)
    n = tuple(int(v) for v in n)
    idx = np.indices(n).reshape(3, -1).T.astype(float)
    o = (np.arange(sub) + 0.5) / sub
    shifts = np.array([(i, j, l) for i in (-1, 0, 1) for j in (-1, 0, 1) for l in (-1, 0, 1)], float)
    inside = np.zeros(idx.shape[0])
    for d in np.array([(a, b, c) for a in o for b in o for c in o]):
        s = (idx + d) / np.array(n, float)
        dist = np.full(s.shape[0], np.inf)
        for sh in shifts:
            dist = np.minimum(dist, np.linalg.norm((s - sh) @ A.T, axis=1))
        inside += dist <= r
    return (inside / sub ** 3).reshape(n)


def sphere_scan(vfs=None, n: int = 24, M: int = 3, nk: int = 31, lattices=("sc", "bcc", "fcc")) -> list[Workload]:
    """The sphere-inclusion volume-fraction scans of the paper's note on normalized band gaps:
    for each lattice, one tungsten-carbide sphere per primitive cell in epoxy (the paper's
    constants) at every volume fraction in vfs (default 0.05 to 0.70 in steps of 0.05), n^3 voxels,
    cutoff M, nk points along the high-symmetry path, 8 bands for gap(6,7)."""
    if vfs is None:
        vfs = [round(0.05 * i, 2) for i in range(1, 15)]
    out = []
    for lat in lattices:
        Q = kpath(lat, nk)
        for vf in vfs:
            rho = sphere_inclusion(lat, (n, n, n), vf)
            out.append(Workload(f"{lat}{n}_M{M}_sphere_vf{vf:.2f}", lat, (n, n, n), M, 8, Q, rho, 1.0, (6,), 0,
                                1.0, dict(PAPER_WC), dict(PAPER_EPOXY)))
    return out
