"""Pins of the oracle's smooth (KS) gap: limit, bounds, derivative, degenerate clusters."""
import numpy as np

from oracle import gap as og


def _table(seed, nk=17, nb=6):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(0.2, 3.0, size=(nk, nb)), axis=1)
    lam[:, 3:] += 1.5  # a clear gap between bands 3 and 4
    return lam


def test_ks_gap_tends_to_the_exact_gap():
    lam = _table(1)
    exact = og.gap(lam, 3).gap
    for beta, tol in ((1e3, 1e-2), (1e5, 1e-4)):
        r = og.ks_gap(lam, 3, beta, omega_ref=1.0)
        assert r.gap <= exact + 1e-15          # a >= max, b <= min
        assert exact - r.gap <= tol * exact


def test_ks_bounds():
    lam = _table(2)
    r = og.ks_gap(lam, 3, 30.0, omega_ref=1.0)
    assert r.lower >= np.sqrt(lam[:, 2]).max()
    assert r.upper <= np.sqrt(lam[:, 3]).min()


def test_ks_weights_match_central_differences():
    lam = _table(3)
    beta, wref = 25.0, 1.7
    r = og.ks_gap(lam, 3, beta, omega_ref=wref)
    h = 1e-6
    for k, b in [(0, 2), (5, 2), (9, 3), (16, 3), (4, 0)]:
        lp, lm = lam.copy(), lam.copy()
        lp[k, b] += h
        lm[k, b] -= h
        fd = (og.ks_gap(lp, 3, beta, wref).gap - og.ks_gap(lm, 3, beta, wref).gap) / (2 * h)
        assert abs(fd - r.weights[k, b]) <= 1e-6 * max(1.0, abs(r.weights).max()), (k, b, fd, r.weights[k, b])


def test_ks_degenerate_cluster_shares_the_weight():
    lam = _table(4)
    lam[7, 1] = lam[7, 2]  # band 3 (index 2) degenerate with band 2 at k = 7
    r = og.ks_gap(lam, 3, 10.0, omega_ref=1.0)
    assert r.weights[7, 1] == r.weights[7, 2] != 0.0
    # the cluster's total equals the single-band weight of the mean eigenvalue
    lam2 = lam.copy()
    r2 = og.ks_gap(lam2, 3, 10.0, omega_ref=1.0, rel_tol=0.0)
    assert np.isclose(r.weights[7, 1] + r.weights[7, 2], r2.weights[7, 2] + r2.weights[7, 1])
