"""Pins of the oracle against exact invariants of the discrete problem (CPU only)."""
import numpy as np
import pytest

import workloads as wl
from oracle import mixed

PH1, PH0 = wl.TUNGSTEN_CARBIDE, wl.EPOXY


def _problem(lattice, n, M, rho, penal=1.0):
    return mixed.build(lattice, n, M, rho, PH1, PH0, penal)


@pytest.mark.parametrize("lattice", ["sc", "bcc", "fcc"])
def test_gamma_has_three_zero_modes(lattice):
    rng = np.random.default_rng(11)
    P = _problem(lattice, (5, 5, 5), 1, rng.uniform(0, 1, (5, 5, 5)), 3.0)
    lam = mixed.bands(P, [[0.0, 0.0, 0.0]], 6)[0]
    scale = lam[3]
    assert np.all(np.abs(lam[:3]) <= 1e-12 * scale)
    assert lam[3] > 1e-6 * scale


def test_operators_hermitian_and_bounded():
    """A = H Phi^-1 H^H is Hermitian PSD; Omega is HPD with spectrum inside V [min rho, max rho]."""
    rng = np.random.default_rng(12)
    P = _problem("fcc", (6, 6, 6), 1, rng.uniform(0, 1, (6, 6, 6)), 3.0)
    A, _ = mixed.operator(P, [0.1, 0.2, 0.3], literal=True)
    assert np.abs(A - A.conj().T).max() <= 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= -1e-12 * ev.max()
    eo = np.linalg.eigvalsh(P.Omega)
    assert eo.min() >= P.V * P.rho_m.min() * (1 - 1e-12)
    assert eo.max() <= P.V * P.rho_m.max() * (1 + 1e-12)


def test_literal_coupling_equals_blockwise():
    """With n_i >= 2M+1 the centroid sum of a non-zero plane-wave difference vanishes, so H is
    block diagonal; the literal dense H and the blockwise contraction give the same operator."""
    rng = np.random.default_rng(13)
    P = _problem("bcc", (5, 6, 7), 2, rng.uniform(0, 1, (5, 6, 7)))
    off = P.I - np.diag(np.diag(P.I))
    assert np.abs(off).max() <= 1e-14
    assert np.allclose(np.diag(P.I), P.V, rtol=1e-14)
    A1, _ = mixed.operator(P, [0.2, -0.1, 0.3], literal=True)
    A2, _ = mixed.operator(P, [0.2, -0.1, 0.3], literal=False)
    assert np.abs(A1 - A2).max() <= 1e-12 * np.abs(A1).max()


def test_time_reversal():
    rng = np.random.default_rng(14)
    P = _problem("fcc", (5, 5, 5), 1, rng.uniform(0, 1, (5, 5, 5)))
    Q = np.array([0.13, 0.31, -0.22])
    l1 = mixed.bands(P, [Q], 8)[0]
    l2 = mixed.bands(P, [-Q], 8)[0]
    assert np.allclose(l1, l2, rtol=1e-11)


def test_translation_invariance():
    rng = np.random.default_rng(15)
    rho = rng.uniform(0, 1, (6, 5, 7))
    Q = np.array([0.21, 0.05, 0.37])
    l1 = mixed.bands(_problem("sc", rho.shape, 1, rho), [Q], 8)[0]
    l2 = mixed.bands(_problem("sc", rho.shape, 1, np.roll(rho, (1, 2, 3), axis=(0, 1, 2))), [Q], 8)[0]
    assert np.allclose(l1, l2, rtol=1e-11)


def test_sc_point_group():
    """SC with n0 = n1 = n2: an axis permutation and a mirror of the design, applied together
    with the same operation on k, leave the bands unchanged."""
    rng = np.random.default_rng(16)
    rho = rng.uniform(0, 1, (5, 5, 5))
    Q = np.array([0.11, 0.27, 0.42])
    base = mixed.bands(_problem("sc", rho.shape, 1, rho), [Q], 8)[0]
    perm = mixed.bands(_problem("sc", rho.shape, 1, np.transpose(rho, (1, 2, 0))), [Q[[1, 2, 0]]], 8)[0]
    mirror = mixed.bands(_problem("sc", rho.shape, 1, rho[::-1]), [Q * [-1, 1, 1]], 8)[0]
    assert np.allclose(base, perm, rtol=1e-11)
    assert np.allclose(base, mirror, rtol=1e-11)


def test_fcc_primitive_permutation_and_inversion():
    """Swapping a1 and a2 of the FCC primitive cell is the Cartesian x <-> y reflection; the
    design's first two fractional axes and Q_1, Q_2 swap with it.  Inversion maps s -> -s
    and Q -> -Q; the rotation about the cube diagonal cycles the axes and Q."""
    rng = np.random.default_rng(17)
    rho = rng.uniform(0, 1, (5, 5, 5))
    Q = np.array([0.19, 0.33, 0.07])
    base = mixed.bands(_problem("fcc", rho.shape, 1, rho), [Q], 8)[0]
    swap = mixed.bands(_problem("fcc", rho.shape, 1, np.transpose(rho, (1, 0, 2))), [Q[[1, 0, 2]]], 8)[0]
    inv = mixed.bands(_problem("fcc", rho.shape, 1, rho[::-1, ::-1, ::-1]), [-Q], 8)[0]
    # the 3-fold rotation about the cube diagonal cycles a1, a2, a3
    rot = mixed.bands(_problem("fcc", rho.shape, 1, np.transpose(rho, (1, 2, 0))), [Q[[1, 2, 0]]], 8)[0]
    assert np.allclose(base, swap, rtol=1e-11)
    assert np.allclose(base, inv, rtol=1e-11)
    assert np.allclose(base, rot, rtol=1e-11)


def test_bcc_primitive_point_group():
    """BCC primitive cell a1 = (-1,1,1)/2, a2 = (1,-1,1)/2, a3 = (1,1,-1)/2: the Cartesian
    x <-> y reflection swaps a1 and a2, the cyclic permutation x -> y -> z cycles a1, a2, a3,
    and inversion maps s -> -s.  Each, applied to the design's fractional axes and to Q
    together, leaves the bands unchanged; the design permuted alone does not."""
    rng = np.random.default_rng(19)
    rho = rng.uniform(0, 1, (5, 5, 5))
    Q = np.array([0.17, 0.29, 0.06])

    def lam(r, q):
        return mixed.bands(_problem("bcc", r.shape, 1, r), [q], 8)[0]

    base = lam(rho, Q)
    assert np.allclose(base, lam(np.transpose(rho, (1, 0, 2)), Q[[1, 0, 2]]), rtol=1e-11)
    assert np.allclose(base, lam(np.transpose(rho, (1, 2, 0)), Q[[1, 2, 0]]), rtol=1e-11)
    assert np.allclose(base, lam(rho[::-1, ::-1, ::-1], -Q), rtol=1e-11)
    moved = lam(np.transpose(rho, (1, 2, 0)), Q)
    assert np.max(np.abs(moved - base) / base[-1]) > 1e-6


def test_element_sum_is_k_independent():
    """The element-sum matrices do not depend on the wavevector (Q cancels in K_q - K_p)."""
    rng = np.random.default_rng(18)
    P = _problem("bcc", (5, 5, 5), 1, rng.uniform(0, 1, (5, 5, 5)))
    from oracle import lattice as lat
    K1 = lat.wavevectors(P.T, [0.3, 0.1, 0.2], P.g)
    F1 = np.exp(2j * np.pi * (P.x @ K1.T))
    T1 = mixed.element_sum(F1, P.rho_m * P.ve)
    T0 = P.Omega[: P.N, : P.N]
    assert np.abs(T1 - T0).max() <= 1e-12 * np.abs(T0).max()
