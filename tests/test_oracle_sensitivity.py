"""Pins of the oracle's sensitivities: literal eq. sensitivityew, finite differences, invariances."""
import numpy as np
import pytest

import workloads as wl
from oracle import gap, mixed, sensitivity

PH1, PH0 = wl.TUNGSTEN_CARBIDE, wl.EPOXY


def test_literal_equals_voxel_form():
    """The per-element derivative matrices of eqs. diffOmega / diffPhi inserted in
    eq. sensitivityew (psi = Omega theta) equal the voxel quadratic forms."""
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.1, 0.9, (3, 4, 3))
    P = mixed.build("bcc", rho.shape, 1, rho, PH1, PH0, 3.0)
    Q = np.array([0.1, 0.25, -0.15])
    sol = mixed.solve_k(P, Q, 5, literal=True)
    for b in (0, 3, 4):
        lit = sensitivity.literal(P, Q, sol.lam[b], sol.theta[:, b])
        vox = sensitivity.voxel(P, sol.lam[b], sol.theta[:, b], sol.s[:, b])
        assert np.abs(lit - vox).max() <= 1e-10 * np.abs(vox).max()


def test_eigenvalue_fd():
    """d lambda / d rho_e equals central differences of the eigenvalue itself."""
    rng = np.random.default_rng(22)
    rho = rng.uniform(0.2, 0.8, (4, 4, 4))
    Q = np.array([0.2, 0.1, 0.3])
    P = mixed.build("sc", rho.shape, 1, rho, PH1, PH0, 3.0)
    sol = mixed.solve_k(P, Q, 6)
    b = 4
    assert sol.lam[b + 1] - sol.lam[b] > 1e-3 * sol.lam[b] and sol.lam[b] - sol.lam[b - 1] > 1e-3 * sol.lam[b]
    g = sensitivity.voxel(P, sol.lam[b], sol.theta[:, b], sol.s[:, b])
    h = 1e-6
    for e in rng.choice(rho.size, 6, replace=False):
        rp, rm = rho.copy().ravel(), rho.copy().ravel()
        rp[e] += h
        rm[e] -= h
        lp = mixed.bands(mixed.build("sc", rho.shape, 1, rp.reshape(rho.shape), PH1, PH0, 3.0), [Q], 6)[0][b]
        lm = mixed.bands(mixed.build("sc", rho.shape, 1, rm.reshape(rho.shape), PH1, PH0, 3.0), [Q], 6)[0][b]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * np.abs(g).max()


def _gap_and_grad(w, rho, n_lower, ks=None):
    P = mixed.build(w.lattice, w.n, w.M, rho, w.phase1, w.phase0, w.penal)
    Q = w.Q if ks is None else w.Q[ks]
    lam, sols = mixed.bands(P, Q, w.nbands, keep=True)
    r = gap.gap(lam, n_lower)
    return r, sensitivity.weighted(P, sols, r.weights)


def test_gap_gradient_fd_sc8_cube():
    """Whole-objective gradient vs central differences on the 8^3 SC cell (p = 1), binary cube
    perturbed by seeded noise so that no degeneracy sits on the extremal bands."""
    w = wl.sc8_binary_cube()
    rng = np.random.default_rng(23)
    rho = np.clip(0.1 + 0.8 * w.rho + 0.05 * rng.standard_normal(w.rho.shape), 0.0, 1.0)
    r, g = _gap_and_grad(w, rho, 3)
    h = 1e-6
    for e in rng.choice(rho.size, 5, replace=False):
        rp, rm = rho.ravel().copy(), rho.ravel().copy()
        rp[e] += h
        rm[e] -= h
        fp = _gap_and_grad(w, rp.reshape(w.n), 3)[0].gap
        fm = _gap_and_grad(w, rm.reshape(w.n), 3)[0].gap
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[e]) <= 2e-5 * np.abs(g).max(), (e, fd, g[e])


@pytest.mark.slow
def test_gap_gradient_fd_sc16_grf():
    """SC 16^3 random field (p = 3): gap(6,7) gradient vs central differences, step 1e-6, on
    20 seeded elements.  The difference quotient re-solves only the two extremal wavevectors,
    which stay extremal under a 1e-6 perturbation."""
    w = wl.sc16_grf()
    rho = w.rho
    r, g = _gap_and_grad(w, rho, 6)
    ks = [r.k_lower, r.k_upper]
    rng = np.random.default_rng(w.seed)
    h = 1e-6
    errs = []
    for e in rng.choice(rho.size, 20, replace=False):
        rp, rm = rho.ravel().copy(), rho.ravel().copy()
        rp[e] += h
        rm[e] -= h
        fp = _gap_and_grad(w, rp.reshape(w.n), 6, ks)[0].gap
        fm = _gap_and_grad(w, rm.reshape(w.n), 6, ks)[0].gap
        errs.append(abs((fp - fm) / (2 * h) - g[e]))
    assert max(errs) <= 1e-5 * np.abs(g).max()


def test_translation_moves_gradient():
    rng = np.random.default_rng(24)
    rho = rng.uniform(0.2, 0.8, (5, 4, 6))
    Q = np.array([0.3, 0.2, 0.1])
    P1 = mixed.build("sc", rho.shape, 1, rho, PH1, PH0, 3.0)
    P2 = mixed.build("sc", rho.shape, 1, np.roll(rho, (2, 1, 3), axis=(0, 1, 2)), PH1, PH0, 3.0)
    s1, s2 = mixed.solve_k(P1, Q, 5), mixed.solve_k(P2, Q, 5)
    g1 = sensitivity.voxel(P1, s1.lam[4], s1.theta[:, 4], s1.s[:, 4]).reshape(rho.shape)
    g2 = sensitivity.voxel(P2, s2.lam[4], s2.theta[:, 4], s2.s[:, 4]).reshape(rho.shape)
    assert np.allclose(np.roll(g1, (2, 1, 3), axis=(0, 1, 2)), g2, rtol=1e-8, atol=1e-10 * np.abs(g1).max())


def test_inversion_maps_gradient():
    """Element derivative matrices at -x are the transposes of those at x, so inverting the
    design (and k) inverts the sensitivity field."""
    rng = np.random.default_rng(25)
    rho = rng.uniform(0.2, 0.8, (5, 5, 5))
    Q = np.array([0.15, 0.1, 0.35])
    P1 = mixed.build("fcc", rho.shape, 1, rho, PH1, PH0, 3.0)
    P2 = mixed.build("fcc", rho.shape, 1, rho[::-1, ::-1, ::-1], PH1, PH0, 3.0)
    s1, s2 = mixed.solve_k(P1, Q, 5), mixed.solve_k(P2, -Q, 5)
    g1 = sensitivity.voxel(P1, s1.lam[4], s1.theta[:, 4], s1.s[:, 4]).reshape(rho.shape)
    g2 = sensitivity.voxel(P2, s2.lam[4], s2.theta[:, 4], s2.s[:, 4]).reshape(rho.shape)
    assert np.allclose(g1[::-1, ::-1, ::-1], g2, rtol=1e-8, atol=1e-10 * np.abs(g1).max())


def test_lattice_mirror_maps_gradient():
    """FCC with a1 and a2 swapped is the Cartesian x <-> y mirror: with the design's first two
    fractional axes and Q_1, Q_2 swapped, the eigenvalue is unchanged and its sensitivity field
    swaps the same two axes (a transposed operand in the field synthesis would break this)."""
    rng = np.random.default_rng(27)
    rho = rng.uniform(0.2, 0.8, (5, 5, 5))
    Q = np.array([0.21, 0.06, -0.13])
    P1 = mixed.build("fcc", rho.shape, 1, rho, PH1, PH0, 3.0)
    P2 = mixed.build("fcc", rho.shape, 1, np.transpose(rho, (1, 0, 2)), PH1, PH0, 3.0)
    s1, s2 = mixed.solve_k(P1, Q, 5), mixed.solve_k(P2, Q[[1, 0, 2]], 5)
    b = 4
    assert abs(s1.lam[b] - s2.lam[b]) <= 1e-11 * s1.lam[b]
    assert s1.lam[b] - s1.lam[b - 1] > 1e-3 * s1.lam[b]
    g1 = sensitivity.voxel(P1, s1.lam[b], s1.theta[:, b], s1.s[:, b]).reshape(rho.shape)
    g2 = sensitivity.voxel(P2, s2.lam[b], s2.theta[:, b], s2.s[:, b]).reshape(rho.shape)
    assert np.allclose(np.transpose(g1, (1, 0, 2)), g2, rtol=1e-8, atol=1e-10 * np.abs(g1).max())
    assert not np.allclose(g1, g2, rtol=1e-3)   # the field is not symmetric by itself


def test_cluster_sum_is_basis_independent():
    """A degenerate pair at a high-symmetry point: the summed sensitivity is unchanged by a
    unitary rotation inside the pair."""
    w = wl.sc8_binary_cube()
    P = mixed.from_workload(w)
    Q = w.Q[-1]  # R point of the symmetric cube inclusion
    sol = mixed.solve_k(P, Q, 6)
    lam = sol.lam
    pairs = [b for b in range(5) if abs(lam[b + 1] - lam[b]) <= 1e-9 * lam[b] and lam[b] > 0]
    assert pairs
    b = pairs[0]
    th = sol.theta[:, b:b + 2]
    ss = sol.s[:, b:b + 2]
    rng = np.random.default_rng(26)
    Z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    U, _ = np.linalg.qr(Z)
    th2, ss2 = th @ U, ss @ U
    g1 = sum(sensitivity.voxel(P, lam[b], th[:, j], ss[:, j]) for j in range(2))
    g2 = sum(sensitivity.voxel(P, lam[b], th2[:, j], ss2[:, j]) for j in range(2))
    assert np.allclose(g1, g2, rtol=1e-9, atol=1e-12 * np.abs(g1).max())
