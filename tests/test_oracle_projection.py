"""Pins of the design-parametrisation oracle (reduced field, Heaviside projection, SC mirror
symmetry; Methods, "Topology optimization formulation"; Results, "Topology optimized
structures"), CPU only:

* the projection's closed forms: H(0) = 0, H(1) = 1, H -> mu as beta -> 0, H -> step as
  beta -> infinity, and its derivative against central differences;
* the filter is a partition of unity (a uniform field passes unchanged), non-negative, and
  covariant under periodic translation of the design grid and under the SC reflections;
* a mirror-expanded octant design gives a reflection-symmetric density;
* the folding of gradients is the adjoint of the mirror expansion (dot-product test), and the
  whole backward map is the adjoint of the linearised forward map;
* the gradient of the projected gap (the adjoint of the band problem chained through the map)
  against central differences of the projected gap itself.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import gap as ogap
from oracle import mixed, projection, sensitivity


@pytest.mark.parametrize("beta", [1.0, 8.0, 64.0])
def test_heaviside_closed_forms(beta):
    assert projection.heaviside(0.0, beta) == 0.0
    assert abs(projection.heaviside(1.0, beta) - 1.0) <= 1e-15
    mu = np.linspace(0.0, 1.0, 41)
    h = 1e-6
    fd = (projection.heaviside(mu + h, beta) - projection.heaviside(mu - h, beta)) / (2 * h)
    assert np.allclose(projection.dheaviside(mu, beta), fd, rtol=1e-6, atol=1e-8)
    assert np.all(np.diff(projection.heaviside(mu, beta)) >= 0) and np.all(projection.dheaviside(mu, beta) > 0)


def test_heaviside_limits():
    mu = np.linspace(0.0, 1.0, 21)
    assert np.allclose(projection.heaviside(mu, 1e-9), mu, atol=1e-8)      # beta -> 0: identity
    big = projection.heaviside(mu, 400.0)
    assert np.allclose(big[mu >= 0.05], 1.0, atol=1e-8) and big[0] == 0.0  # beta -> inf: step


@pytest.mark.parametrize("lattice,n,spacing,rad", [("sc", (8, 8, 8), 2, 2.5), ("bcc", (6, 6, 6), 2, 2.2),
                                                   ("fcc", (6, 4, 8), 2, 2.0), ("sc", (6, 6, 6), 1, 1.6)])
def test_filter_partition_of_unity_and_translation(lattice, n, spacing, rad):
    A = mixed.lat.primitive_vectors(lattice)
    r = rad * np.linalg.norm(A[:, 0]) / n[0]
    F = projection.filter_matrix(lattice, n, spacing, r)
    assert np.all(F >= 0.0)
    assert np.allclose(F.sum(axis=1), 1.0, atol=1e-14)
    nd, _ = projection.design_grid(n, spacing)
    rng = np.random.default_rng(11)
    phi = rng.uniform(size=nd)
    mu = (F @ phi.ravel()).reshape(n)
    for ax in range(3):  # rolling the nodes by one rolls the elements by `spacing`
        mu2 = (F @ np.roll(phi, 1, axis=ax).ravel()).reshape(n)
        assert np.allclose(mu2, np.roll(mu, spacing, axis=ax), atol=1e-14)


def test_filter_reflection_covariance_sc():
    n, spacing = (8, 8, 8), 2
    F = projection.filter_matrix("sc", n, spacing, 2.5 / 8)
    nd, _ = projection.design_grid(n, spacing)
    phi = np.random.default_rng(12).uniform(size=nd)
    mu = (F @ phi.ravel()).reshape(n)
    for ax in range(3):
        mu2 = (F @ np.flip(phi, axis=ax).ravel()).reshape(n)
        assert np.allclose(mu2, np.flip(mu, axis=ax), atol=1e-14)


def test_mirror_expansion_symmetry_and_adjoint():
    nd = (6, 6, 6)
    rng = np.random.default_rng(13)
    x = rng.uniform(size=27)
    full = projection.mirror_expand(x, nd).reshape(nd)
    for ax in range(3):
        assert np.array_equal(full, np.flip(full, axis=ax))
    assert np.array_equal(full[:3, :3, :3].ravel(), x)
    g = rng.standard_normal(nd)
    assert abs(np.dot(full.ravel(), g.ravel()) - np.dot(x, projection.mirror_fold(g, nd))) <= 1e-12


@pytest.mark.parametrize("octant", [False, True])
def test_backward_is_adjoint_of_linearised_forward(octant):
    dm = projection.DesignMap("sc", (8, 8, 8), spacing=2, radius=2.5 / 8, octant=octant)
    rng = np.random.default_rng(14)
    x = rng.uniform(0.1, 0.9, dm.nvars)
    dx = rng.standard_normal(dm.nvars)
    g = rng.standard_normal(dm.n)
    beta = 6.0
    h = 1e-6
    fd = (np.sum(g * dm.forward(x + h * dx, beta)) - np.sum(g * dm.forward(x - h * dx, beta))) / (2 * h)
    assert abs(fd - np.dot(dm.backward(x, beta, g), dx)) <= 1e-7 * abs(fd)
    if octant:
        rho = dm.forward(x, beta)
        for ax in range(3):
            assert np.allclose(rho, np.flip(rho, axis=ax), atol=1e-15)


def test_default_radius_reading():
    """1.4 element edges: on the paper's 24^3 SC mesh with nodes every 2 elements, every element
    sees exactly the node of its own 2 x 2 x 2 block (sqrt(3)/2 = 0.87 edges away; the next nodes
    are 1.66 edges away), so the reduced field is block-constant there."""
    dm = projection.DesignMap("sc", (24, 24, 24), spacing=2)
    assert np.all(np.count_nonzero(dm.F, axis=1) == 1)


def test_projected_gap_gradient_central_differences():
    """SC 8^3 cell, M = 1, octant-symmetric reduced field (4^3 nodes, 8 free variables), radius
    2.5 edges, beta = 4: d gap(3,4) / dx from the adjoint chained through the map against central
    differences (step 1e-5) of the projected gap on every variable."""
    w = wl.sc8_binary_cube()
    dm = projection.DesignMap("sc", w.n, spacing=2, radius=2.5 / 8, octant=True)
    rng = np.random.default_rng(15)
    x = rng.uniform(0.2, 0.8, dm.nvars)
    beta = 4.0

    def gap_of(xv, grad=False):
        rho = dm.forward(xv, beta)
        P = mixed.build(w.lattice, w.n, w.M, rho, w.phase1, w.phase0, 1.0)
        lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
        r = ogap.gap(lam, 3)
        if not grad:
            return r.gap
        g_rho = sensitivity.weighted(P, sols, r.weights)
        return r.gap, dm.backward(xv, beta, g_rho)

    _, g = gap_of(x, grad=True)
    h = 1e-5
    fd = np.array([(gap_of(x + h * e) - gap_of(x - h * e)) / (2 * h) for e in np.eye(dm.nvars)])
    assert np.allclose(g, fd, rtol=1e-4, atol=1e-6 * np.abs(fd).max()), (g, fd)
