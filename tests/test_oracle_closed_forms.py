"""Pins of the oracle against closed forms and the paper's printed numbers (CPU only)."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import brentq

import workloads as wl
from oracle import gap, lattice as lat, mixed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _speeds(phase):
    E, nu, rho = phase["E"], phase["nu"], phase["rho"]
    mu = E / (2 * (1 + nu))
    lam_l = E * nu / ((1 + nu) * (1 - 2 * nu))
    return np.sqrt((lam_l + 2 * mu) / rho), np.sqrt(mu / rho)


@pytest.mark.parametrize("lattice", ["sc", "bcc", "fcc"])
@pytest.mark.parametrize("M", [1, 2])
def test_homogeneous_medium_is_exact(lattice, M):
    """In a homogeneous cell the method is exact: lambda = (2 pi)^2 |K_p|^2 c^2 with c_L once
    and c_T twice per plane wave (omega = c |k + G|)."""
    w = wl.homogeneous(lattice, (2 * M + 2,) * 3, M, 14, 12 if lattice != "fcc" else 14, value=1.0)
    P = mixed.from_workload(w)
    cL, cT = _speeds(w.phase1)
    for Q in w.Q[::4]:
        lam = mixed.bands(P, [Q], 14)[0]
        K = lat.wavevectors(P.T, Q, P.g)
        k2 = (2 * np.pi) ** 2 * np.sum(K * K, axis=1)
        ref = np.sort(np.concatenate([k2 * cL ** 2, k2 * cT ** 2, k2 * cT ** 2]))[:14]
        assert np.max(np.abs(lam - ref)) <= 1e-12 * ref.max()


def test_homogeneous_mixture_uses_interpolated_compliance():
    """rho_e = 0.5, p = 1: density and compliance are the phase averages; the speeds follow
    from the averaged compliance (bulk 1/(3 f1), shear 1/(2 f2))."""
    w = wl.homogeneous("sc", (4, 4, 4), 1, 9, 8, value=0.5)
    P = mixed.from_workload(w)
    p1, p0 = w.phase1, w.phase0
    f1 = 0.5 * ((1 - 2 * p1["nu"]) / p1["E"] + (1 - 2 * p0["nu"]) / p0["E"])
    f2 = 0.5 * ((1 + p1["nu"]) / p1["E"] + (1 + p0["nu"]) / p0["E"])
    rho = 0.5 * (p1["rho"] + p0["rho"])
    Kb, mu = 1 / (3 * f1), 1 / (2 * f2)
    cL2, cT2 = (Kb + 4 * mu / 3) / rho, mu / rho
    Q = w.Q[2]
    K = lat.wavevectors(P.T, Q, P.g)
    k2 = (2 * np.pi) ** 2 * np.sum(K * K, axis=1)
    ref = np.sort(np.concatenate([k2 * cL2, k2 * cT2, k2 * cT2]))[:9]
    lam = mixed.bands(P, [Q], 9)[0]
    assert np.allclose(lam, ref, rtol=1e-12, atol=1e-12 * ref.max())



def _mixture_speeds2(p1, p0, chi):
    """Squared longitudinal and transverse speeds of the uniform mixture whose density and
    compliance moduli f1 = (1 - 2 nu)/E, f2 = (1 + nu)/E are linear in chi."""
    f1 = (1 - 2 * p0["nu"]) / p0["E"] + chi * ((1 - 2 * p1["nu"]) / p1["E"] - (1 - 2 * p0["nu"]) / p0["E"])
    f2 = (1 + p0["nu"]) / p0["E"] + chi * ((1 + p1["nu"]) / p1["E"] - (1 + p0["nu"]) / p0["E"])
    rho = p0["rho"] + chi * (p1["rho"] - p0["rho"])
    Kb, mu = 1 / (3 * f1), 1 / (2 * f2)
    return (Kb + 4 * mu / 3) / rho, mu / rho


def test_uniform_mixture_power_law_p3():
    """rho_e = 0.5 everywhere with p = 3: the material is the mixture at chi = 0.5^3 = 0.125
    (not at rho = 0.5), and a uniform change of rho moves every eigenvalue by
    d lambda/d chi * d chi/d rho with d chi/d rho = 3 * 0.5^2 = 0.75.  The element sensitivities
    of one eigenpair therefore sum to that closed form; checked on the two transverse modes and the
    longitudinal mode of the lowest plane wave at a generic wavevector (a wrong exponent, or chi
    and d chi both taken linear, fails it)."""
    from oracle import sensitivity
    w = wl.homogeneous("sc", (4, 4, 4), 1, 9, 8, value=0.5)
    w.penal = 3.0
    P = mixed.from_workload(w)
    assert np.allclose(P.chi, 0.125) and np.allclose(P.dchi, 0.75)
    Q = np.array([0.13, 0.07, 0.21])   # generic: one shortest K, its modes apart from the rest
    K = lat.wavevectors(P.T, Q, P.g)
    k2 = (2 * np.pi) ** 2 * np.sum(K * K, axis=1)
    cL2, cT2 = _mixture_speeds2(w.phase1, w.phase0, 0.125)
    ref = np.sort(np.concatenate([k2 * cL2, k2 * cT2, k2 * cT2]))[:9]
    lam, sols = mixed.bands(P, [Q], 9, keep=True)
    assert np.allclose(lam[0], ref, rtol=1e-12, atol=1e-12 * ref.max())
    # closed-form derivative along chi of the modes of the lowest plane wave (central difference
    # of the closed form itself, exact to ~1e-10 for these smooth rational functions)
    kmin = np.min(k2)
    h = 1e-6
    sp = _mixture_speeds2(w.phase1, w.phase0, 0.125 + h), _mixture_speeds2(w.phase1, w.phase0, 0.125 - h)
    dL = kmin * (sp[0][0] - sp[1][0]) / (2 * h)
    dT = kmin * (sp[0][1] - sp[1][1]) / (2 * h)
    bL = int(np.argmin(np.abs(lam[0] - kmin * cL2)))   # the longitudinal mode, wherever it sorts
    assert abs(lam[0][bL] - kmin * cL2) <= 1e-12 * ref.max()
    assert np.all(np.abs(np.delete(lam[0], bL) - lam[0][bL]) > 1e-6 * lam[0][bL])  # isolated
    sol = sols[0]
    for b, d in ((0, dT), (1, dT), (bL, dL)):
        total = np.sum(sensitivity.voxel(P, sol.lam[b], sol.theta[:, b], sol.s[:, b]))
        assert abs(total - 0.75 * d) <= 1e-7 * abs(0.75 * d), (b, total, 0.75 * d)


def _rytov_roots(k, d1, d2, c1, c2, Z1, Z2, wmax, count):
    def f(w):
        return (np.cos(w * d1 / c1) * np.cos(w * d2 / c2)
                - 0.5 * (Z1 / Z2 + Z2 / Z1) * np.sin(w * d1 / c1) * np.sin(w * d2 / c2) - np.cos(k))
    ws = np.linspace(1e-9, wmax, 20001)
    fs = f(ws)
    roots = [brentq(f, ws[i], ws[i + 1]) for i in range(len(ws) - 1) if fs[i] * fs[i + 1] < 0]
    return np.array(roots[:count])


def test_laminate_converges_to_rytov():
    """SC cell layered along x, k along x: the lowest pressure and shear bands approach the
    exact Rytov dispersion relation of the periodic bilayer as the cutoff M grows."""
    frac = 0.5
    kx = 0.3
    p1, p0 = wl.TUNGSTEN_CARBIDE, wl.EPOXY
    (cL1, cT1), (cL0, cT0) = _speeds(p1), _speeds(p0)
    errs = []
    for M in (1, 2, 3):
        w = wl.laminate(48, 2 * M + 1, M, frac, [kx])
        P = mixed.from_workload(w)
        lam = mixed.bands(P, w.Q, 6)[0]
        om = np.sqrt(lam)
        k = 2 * np.pi * kx
        rs = _rytov_roots(k, frac, 1 - frac, cT1, cT0, p1["rho"] * cT1, p0["rho"] * cT0, 3e4, 1)
        rp = _rytov_roots(k, frac, 1 - frac, cL1, cL0, p1["rho"] * cL1, p0["rho"] * cL0, 3e4, 1)
        # lowest three modes at this k: the shear pair and the pressure mode
        ref = np.sort([rs[0], rs[0], rp[0]])
        errs.append(np.max(np.abs(om[:3] - ref) / ref))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 2e-2


def test_laminate_optimum_matches_paper():
    """The paper's 1-D optimum (first gap of a WC/epoxy bilayer, maximal at WC fraction 0.737)
    from the exact Rytov relation at the zone boundary k d = pi, gap in the omega form through
    the oracle's gap function.  Waves of speed sqrt(E/rho) (rod) and shear waves both give the
    printed value within 0.4 points and peak within 0.005 of the printed fraction; pressure waves
    peak at 154.5 % near 0.724, so the printed scan is not of pressure waves."""
    c = json.load(open(os.path.join(GOLDEN, "paper_laminate_optimum.json")))
    p1, p0 = wl.PAPER_WC, wl.PAPER_EPOXY
    (cL1, cT1), (cL0, cT0) = _speeds(p1), _speeds(p0)
    rod1, rod0 = np.sqrt(p1["E"] / p1["rho"]), np.sqrt(p0["E"] / p0["rho"])

    def first_gap(f, c1, c0):
        edges = _rytov_roots(np.pi, f, 1 - f, c1, c0, p1["rho"] * c1, p0["rho"] * c0, 2.0e5, 2)
        return gap.gap((edges[None, :] ** 2), 1, gap.MODE_OMEGA).gap * 100

    fs = np.arange(0.700, 0.7705, 0.005)
    for c1, c0 in ((rod1, rod0), (cT1, cT0)):
        assert abs(first_gap(c["volume_fraction"], c1, c0) - c["printed_gap_pct"]) <= 0.4
        g = [first_gap(f, c1, c0) for f in fs]
        assert abs(fs[int(np.argmax(g))] - c["volume_fraction"]) <= 0.005 + 1e-9
    gp = [first_gap(f, cL1, cL0) for f in fs]
    assert abs(max(gp) - c["printed_gap_pct"]) > 0.8


def test_gap_matches_paper_band_edges():
    """The omega form of the gap reproduces the percentages printed with the paper's band edges."""
    cases = json.load(open(os.path.join(GOLDEN, "paper_band_edges.json")))["cases"]
    for c in cases:
        lam = (2 * np.pi * 1e3 * np.array([[c["lower_khz"], c["upper_khz"]]])) ** 2
        g = gap.gap(lam, 1, gap.MODE_OMEGA).gap * 100
        if c["consistent"]:
            assert abs(g - c["printed_gap_pct"]) < 0.006, c
        else:
            assert abs(g - c["omega_form_pct"]) < 0.006, c
        g_lambda = gap.gap(lam, 1, gap.MODE_LAMBDA).gap * 100
        assert abs(g_lambda - c["printed_gap_pct"]) > 10.0


def test_sphere_inclusion_gaps_match_paper():
    """Tungsten-carbide spheres in epoxy with the paper's constants, one per primitive cell, at
    the volume fractions where the paper's scans peak: gap(6,7) lies within 3 percentage points
    of the printed maxima at M = 3, the cutoff of the paper's optimization runs.  The pin is
    approximate because the paper states neither the cutoff nor the grid of these scans, and
    the cutoff alone moves the BCC and FCC gaps by 3-5 points between M = 3 and M = 4.  Other
    constants (the stiffer WC of the benchmark workloads) or a 20 % heavier inclusion move the
    gap by 2-7 points; swapping the phases closes it.  Only the distinct high-symmetry points
    are sampled: for these designs the gap edges sit there (within 0.1 point of a 31-point
    boundary path)."""
    cases = json.load(open(os.path.join(GOLDEN, "paper_sphere_inclusions.json")))["cases"]
    n = (24, 24, 24)
    got = {}
    for c in cases:
        rho = wl.sphere_inclusion(c["lattice"], n, c["volume_fraction"])
        assert abs(rho.mean() - c["volume_fraction"]) < 2e-3
        P = mixed.build(c["lattice"], n, 3, rho, wl.PAPER_WC, wl.PAPER_EPOXY, 1.0)
        lam = mixed.bands(P, wl.high_symmetry_points(c["lattice"]), 8)
        got[c["lattice"]] = gap.gap(lam, 6).gap * 100
        assert abs(got[c["lattice"]] - c["printed_gap_pct"]) <= 3.0, (c, got)
    assert min(got["bcc"], got["fcc"]) > got["sc"] + 20.0


def test_gap_weights_are_the_gradient_of_the_gap():
    rng = np.random.default_rng(5)
    lam = np.sort(rng.uniform(1.0, 9.0, size=(7, 5)), axis=1)
    lam[:, 3:] += 6.0
    for mode in (gap.MODE_OMEGA, gap.MODE_LAMBDA):
        r = gap.gap(lam, 3, mode)
        h = 1e-6
        for k in range(7):
            for b in range(5):
                lp, lm = lam.copy(), lam.copy()
                lp[k, b] += h
                lm[k, b] -= h
                fd = (gap.gap(lp, 3, mode).gap - gap.gap(lm, 3, mode).gap) / (2 * h)
                assert abs(fd - r.weights[k, b]) < 1e-6 * max(1.0, abs(fd))


def test_gap_ties_take_lowest_k_and_clusters_share_weight():
    lam = np.array([[1.0, 2.0, 5.5, 6.0], [1.0, 2.0, 5.0, 5.0], [1.0, 2.0, 5.0, 5.0]])
    r = gap.gap(lam, 2, gap.MODE_LAMBDA)
    assert r.k_upper == 1
    assert r.weights[1, 2] == r.weights[1, 3] != 0.0
    assert r.weights[2].sum() == 0.0
