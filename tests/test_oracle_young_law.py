"""Pins of the oracle's Young's-modulus interpolation (eq. combinematerial read literally: E and
nu linear in chi, each element the compliance of its interpolated isotropic material)."""
import numpy as np

import workloads as wl
from oracle import lattice as lat
from oracle import mixed, sensitivity

PH1, PH0 = wl.TUNGSTEN_CARBIDE, wl.EPOXY


def test_pure_phases_agree_with_the_compliance_law():
    """At rho = 0 and 1 both laws give the pure phases, up to the rounding of D0 + (D1 - D0)."""
    for value in (0.0, 1.0):
        rho = np.full((4, 4, 4), value)
        Pc = mixed.build("fcc", rho.shape, 1, rho, PH1, PH0, 1.0)
        Py = mixed.build("fcc", rho.shape, 1, rho, PH1, PH0, 1.0, law="young")
        assert np.abs(Py.Phi - Pc.Phi).max() <= 1e-14 * np.abs(Pc.Phi).max()
        assert np.array_equal(Py.Omega, Pc.Omega)


def test_uniform_mixture_is_the_interpolated_material():
    """rho_e = 0.3, p = 1: the cell is the homogeneous medium of E(0.3), nu(0.3), rho(0.3);
    its bands are the closed form (2 pi |K|)^2 c^2 for pressure and shear speeds.  The same cell
    under the compliance law is softer (a harmonic rather than arithmetic mean of the moduli)."""
    t = 0.3
    rho = np.full((4, 4, 4), t)
    P = mixed.build("bcc", rho.shape, 1, rho, PH1, PH0, 1.0, law="young")
    E = PH0["E"] + t * (PH1["E"] - PH0["E"])
    nu = PH0["nu"] + t * (PH1["nu"] - PH0["nu"])
    dens = PH0["rho"] + t * (PH1["rho"] - PH0["rho"])
    mu, lam_l = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    cL2, cT2 = (lam_l + 2 * mu) / dens, mu / dens
    Q = np.array([0.2, 0.1, -0.15])
    K = lat.wavevectors(P.T, Q, P.g)
    k2 = (2 * np.pi) ** 2 * np.sum(K * K, axis=1)
    ref = np.sort(np.concatenate([k2 * cL2, k2 * cT2, k2 * cT2]))[:9]
    lam = mixed.bands(P, [Q], 9)[0]
    assert np.allclose(lam, ref, rtol=1e-12, atol=1e-12 * ref.max())
    soft = mixed.bands(mixed.build("bcc", rho.shape, 1, rho, PH1, PH0, 1.0), [Q], 9)[0]
    assert np.all(soft < lam * (1 - 1e-3))


def test_per_element_sensitivity_matches_literal_form_and_differences():
    """With dD/dchi varying per element, the voxel quadratic form equals the literal
    per-element eq. sensitivityew, and both equal central differences of the eigenvalue."""
    rng = np.random.default_rng(26)
    rho = rng.uniform(0.1, 0.9, (3, 4, 3))
    Q = np.array([0.1, 0.25, -0.15])
    P = mixed.build("bcc", rho.shape, 1, rho, PH1, PH0, 3.0, law="young")
    sol = mixed.solve_k(P, Q, 5, literal=True)
    b = 4
    assert sol.lam[b] - sol.lam[b - 1] > 1e-3 * sol.lam[b]
    vox = sensitivity.voxel(P, sol.lam[b], sol.theta[:, b], sol.s[:, b])
    lit = sensitivity.literal(P, Q, sol.lam[b], sol.theta[:, b])
    assert np.abs(lit - vox).max() <= 1e-10 * np.abs(vox).max()
    h = 1e-6
    for e in rng.choice(rho.size, 5, replace=False):
        rp, rm = rho.ravel().copy(), rho.ravel().copy()
        rp[e] += h
        rm[e] -= h
        fp = mixed.bands(mixed.build("bcc", rho.shape, 1, rp.reshape(rho.shape), PH1, PH0, 3.0, law="young"), [Q], 5)[0][b]
        fm = mixed.bands(mixed.build("bcc", rho.shape, 1, rm.reshape(rho.shape), PH1, PH0, 3.0, law="young"), [Q], 5)[0][b]
        assert abs((fp - fm) / (2 * h) - vox[e]) <= 1e-5 * np.abs(vox).max(), e


def test_compliance_derivative_pattern():
    """dD/dchi from the closed form equals central differences of the interpolated compliance."""
    rho = np.linspace(0.05, 0.95, 7)
    _, _, _, D, _, dD = mixed.material_fields(rho, PH1, PH0, 1.0, law="young")
    h = 1e-7
    _, _, _, Dp, _, _ = mixed.material_fields(rho + h, PH1, PH0, 1.0, law="young")
    _, _, _, Dm, _, _ = mixed.material_fields(rho - h, PH1, PH0, 1.0, law="young")
    fd = (Dp - Dm) / (2 * h)
    assert np.abs(fd - dD).max() <= 1e-6 * np.abs(dD).max()
