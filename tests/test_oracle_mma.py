"""Pins of the oracle's box-constrained MMA step: the subproblem's closed-form minimiser, the
model's first-order agreement with the objective, convergence on a separable quadratic with
interior and active bounds, and ascent on the smooth gap of a small cell."""
import numpy as np

import workloads as wl
from oracle import gap as og
from oracle import mixed, mma, sensitivity


def _model(x, p, q, L, U):
    return p / (U - x) + q / (x - L)


def test_subproblem_minimiser_by_brute_force():
    """x* = (sqrt(p) L + sqrt(q) U) / (sqrt(p) + sqrt(q)) minimises p/(U-x) + q/(x-L) on (L, U)."""
    rng = np.random.default_rng(81)
    for _ in range(20):
        L, U = -rng.uniform(0.1, 2.0), rng.uniform(1.0, 3.0)
        p, q = rng.uniform(0.0, 5.0), rng.uniform(0.0, 5.0)
        grid = np.linspace(L, U, 200003)[1:-1]
        xb = grid[np.argmin(_model(grid, p, q, L, U))]
        xs = (np.sqrt(p) * L + np.sqrt(q) * U) / (np.sqrt(p) + np.sqrt(q))
        assert abs(xs - xb) <= 3 * (U - L) / 200000


def test_model_matches_objective_gradient():
    """The convex model's derivative at the current iterate equals the objective's (to minimise,
    dg = -df); a swapped p/q or sign would fail.  Checked through the step's own asymptotes by
    recomputing p, q from the documented rules."""
    rng = np.random.default_rng(82)
    x = rng.uniform(0.05, 0.95, 50)
    df = rng.standard_normal(50)
    st = mma.MMAState()
    L, U = mma.asymptotes(x, st)
    dg = -df
    pos, neg = np.maximum(dg, 0), np.maximum(-dg, 0)
    p = (U - x) ** 2 * (1.001 * pos + 0.001 * neg + 1e-5)
    q = (x - L) ** 2 * (0.001 * pos + 1.001 * neg + 1e-5)
    h = 1e-7
    d = (_model(x + h, p, q, L, U) - _model(x - h, p, q, L, U)) / (2 * h)
    assert np.allclose(d, dg, rtol=1e-6, atol=1e-6)
    # the step moves every variable along the ascent direction of f (or stays at a bound)
    xn = mma.step(x, df, mma.MMAState())
    assert np.all(np.sign(xn - x) == np.sign(df))


def test_converges_on_separable_quadratic():
    """f = -sum (x - c)^2 with some c outside [0, 1]: components whose optimum is outside the
    box land exactly on the bound; the others end within the asymptote floor (0.01 of the box)
    of c.  Plain MMA goes no closer: its step is about 0.9 of the asymptote distance wherever the
    gradient dominates the 1e-5 regulariser, and oscillation shrinks that distance only down
    to the floor, where the iterates settle into a two-cycle around c."""
    rng = np.random.default_rng(83)
    c = rng.uniform(-0.4, 1.4, 40)
    x = np.full(40, 0.5)
    st = mma.MMAState()
    for _ in range(80):
        x = mma.step(x, -2.0 * (x - c), st)
        assert np.all((x >= 0.0) & (x <= 1.0))
    out = (c < 0.0) | (c > 1.0)
    assert np.array_equal(x[out], np.clip(c[out], 0.0, 1.0))
    assert np.abs(x[~out] - c[~out]).max() <= 0.01


def test_steps_raise_the_smooth_gap_of_a_small_cell():
    """Three steps on the smooth omega-form gap(3,4) of the SC 8^3 cube cell (M = 1, ten
    wavevectors), gradient from the oracle's adjoint: the gap grows at every step."""
    w = wl.sc8_binary_cube()
    rng = np.random.default_rng(84)
    rho = np.clip(0.2 + 0.6 * w.rho + 0.05 * rng.standard_normal(w.n), 0.0, 1.0).ravel()
    wref = 2 * np.pi * np.sqrt(w.phase1["E"] / w.phase1["rho"])

    def objective(r):
        P = mixed.build(w.lattice, w.n, w.M, r.reshape(w.n), w.phase1, w.phase0, w.penal)
        lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
        res = og.ks_gap(lam, 3, 50.0, omega_ref=wref)
        return res.gap, sensitivity.weighted(P, sols, res.weights)

    st = mma.MMAState()
    f, g = objective(rho)
    history = [f]
    for _ in range(3):
        rho = mma.step(rho, g, st)
        f, g = objective(rho)
        history.append(f)
    assert all(b > a for a, b in zip(history, history[1:])), history
