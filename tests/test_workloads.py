"""The seeded input generators (CPU): wavevector paths, high-symmetry points, designs, seeds."""
import itertools

import numpy as np
import pytest

import workloads as wl


def _cartesian(lattice, Q):
    """K from reduced coordinates Q_j = K . a_j."""
    return np.asarray(Q) @ np.linalg.inv(wl._primitive(lattice))


def _reciprocal_lattice(lattice, r=2):
    B = np.linalg.inv(wl._primitive(lattice)).T   # columns b_i, b_i . a_j = delta_ij
    return np.array([B @ np.array(g) for g in itertools.product(range(-r, r + 1), repeat=3) if any(g)])


@pytest.mark.parametrize("lattice", ["sc", "bcc", "fcc"])
def test_high_symmetry_points_lie_on_the_zone_boundary(lattice):
    """Every high-symmetry point other than Gamma is on the first Brillouin zone's boundary: as
    close to some reciprocal lattice vector G as to the origin, and closer to none."""
    G = _reciprocal_lattice(lattice)
    K = _cartesian(lattice, wl.high_symmetry_points(lattice))
    for name, k in zip(wl.HIGH_SYMMETRY[lattice], K):
        if name == "G":
            assert np.allclose(k, 0)
            continue
        d = np.linalg.norm(k - G, axis=1)
        assert d.min() >= np.linalg.norm(k) - 1e-12, name
        assert np.isclose(d.min(), np.linalg.norm(k), rtol=1e-12), name


@pytest.mark.parametrize("lattice,nk", [("sc", 10), ("sc", 31), ("bcc", 64), ("fcc", 100), ("fcc", 48)])
def test_kpath_visits_every_vertex_along_straight_segments(lattice, nk):
    Q = wl.kpath(lattice, nk)
    assert Q.shape == (nk, 3)
    K = _cartesian(lattice, Q)
    spec = wl.PATHS[lattice]
    pts = wl.HIGH_SYMMETRY[lattice]
    # the vertices, in order, are a subsequence of the path
    verts = [np.array(pts[v], float) for part in spec.split("|") for v in part.split("-")]
    idx = []
    start = 0
    for v in verts:
        hit = next(i for i in range(start, nk) if np.allclose(K[i], v, atol=1e-12))
        idx.append(hit)
        start = hit + 1
    assert idx[0] == 0 and idx[-1] == nk - 1
    # between consecutive vertices of one polyline the points are collinear and evenly spaced
    bounds = np.cumsum([len(part.split("-")) for part in spec.split("|")])
    for a in range(len(verts) - 1):
        if a + 1 in bounds:   # a jump '|' between polylines
            continue
        seg = K[idx[a]:idx[a + 1] + 1]
        steps = np.diff(seg, axis=0)
        assert np.allclose(steps, steps[0], atol=1e-12)


@pytest.mark.parametrize("lattice,vf", [("sc", 0.2), ("sc", 0.412), ("bcc", 0.545), ("fcc", 0.588), ("fcc", 0.7)])
def test_sphere_inclusion_volume_fraction(lattice, vf):
    rho = wl.sphere_inclusion(lattice, (24, 24, 24), vf)
    assert rho.min() >= 0.0 and rho.max() <= 1.0
    assert abs(rho.mean() - vf) <= 2e-3
    assert np.all(np.isin(rho * 27, np.arange(28)))   # 27 sample points per voxel


def test_sphere_inclusion_has_the_cells_symmetry():
    """A sphere on the lattice points of the SC cell: the voxel occupancies are invariant under
    the cube's axis permutations and mirrors (centroids at (i + 1/2)/n map onto each other)."""
    rho = wl.sphere_inclusion("sc", (16, 16, 16), 0.3)
    for perm in itertools.permutations(range(3)):
        assert np.array_equal(np.transpose(rho, perm), rho)
    assert np.array_equal(rho[::-1], rho)
    # and for FCC the swap of a1 and a2 (a mirror of the cubic lattice)
    rf = wl.sphere_inclusion("fcc", (12, 12, 12), 0.5)
    assert np.array_equal(np.transpose(rf, (1, 0, 2)), rf)


def test_seeded_designs_are_reproducible_and_distinct():
    a, b = wl.sc16_grf(0), wl.sc16_grf(0)
    assert np.array_equal(a.rho, b.rho) and a.seed == b.seed == wl.SEED_BASE["sc16_M2_grf"]
    assert not np.array_equal(wl.sc16_grf(1).rho, a.rho)
    seeds = [w.seed for w in wl.batch32_mixed()]
    seeds += [wl.sc8_binary_cube().seed, a.seed, wl.bcc24_grf().seed, wl.fcc32_levelset().seed]
    assert len(set(seeds)) == len(seeds)


def test_design_generators_statistics():
    rng = np.random.default_rng(5)
    z = wl.gaussian_random_field((16, 16, 16), 1.0 / 6.0, rng)
    assert abs(z.mean()) <= 1e-12 and abs(z.std() - 1.0) <= 1e-12
    w = wl.fcc32_levelset()
    assert w.rho.min() > 0.0 and w.rho.max() < 1.0
    assert abs(np.mean(w.rho > 0.5) - 0.5) <= 1e-3   # thresholded at the median of phi
    for d in wl.batch32_mixed():
        assert min(d.n) >= 2 * d.M + 1 and d.nk == 48 and d.nbands == 20
