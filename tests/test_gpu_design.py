"""GPU parity of the design parametrisation (reduced design field, Heaviside projection, SC octant
mirror symmetry; Methods, "Topology optimization formulation"; Results, "Topology optimized
structures") against the oracle, through the C ABI:

* the projected densities, 1e-14 relative to the largest (the same FP64 sums in another order);
* the chain rule d/dx from a seeded d/drho, 1e-13 relative (L-infinity over the variables);
* the projected gap's gradient end to end (densities from the map, the band and adjoint path,
  the chain rule back) against the oracle's, 1e-5 (FP64 form) and 1e-4 (mixed form) relative L2;
* the optimization loop on free variables with the beta continuation against the oracle's loop.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import gap as ogap
from oracle import mixed, projection, sensitivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("sc", (16, 16, 16), 2, 2.5, True), ("sc", (8, 12, 8), 2, 2.2, False), ("bcc", (12, 12, 12), 2, 2.3, False),
         ("fcc", (12, 12, 16), 2, 2.1, False), ("sc", (10, 10, 10), 1, 1.6, False)]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


def edge(lattice, n):
    return np.linalg.norm(mixed.lat.primitive_vectors(lattice)[:, 0]) / n[0]


@pytest.mark.parametrize("lattice,n,spacing,rad,octant", CASES)
def test_projection_and_chain_rule_match_oracle(B, lattice, n, spacing, rad, octant):
    from paper_1603_06855_gb300.solver import DesignMap
    r = rad * edge(lattice, n)
    ref = projection.DesignMap(lattice, n, spacing=spacing, radius=r, octant=octant)
    dm = DesignMap(lattice, n, spacing=spacing, radius=r, octant=octant)
    assert dm.nvars == ref.nvars
    rng = np.random.default_rng(hash((lattice, n)) % 2**32)
    for beta in (1.0, 16.0):
        x = rng.uniform(0.0, 1.0, ref.nvars)
        rho = dm.project(torch.from_numpy(x), beta).cpu().numpy()
        rho_ref = ref.forward(x, beta)
        assert np.abs(rho - rho_ref).max() <= 1e-14 * np.abs(rho_ref).max()
        g = rng.standard_normal(n)
        gx = dm.backprop(torch.from_numpy(g)).cpu().numpy()
        gx_ref = ref.backward(x, beta, g)
        assert np.abs(gx - gx_ref).max() <= 1e-13 * np.abs(gx_ref).max()
    dm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_projected_gap_gradient_matches_oracle(B, precision):
    """SC 16^3, M = 2, 30 k, octant-symmetric reduced field (8^3 nodes, 64 free variables, radius
    2.5 edges, beta = 4): gap(6,7) and d gap / dx through the autograd chain ProjectFn -> GapFn."""
    from paper_1603_06855_gb300.solver import BandSolver, DesignMap, ProjectFn, gap
    w = wl.sc16_grf()
    r = 2.5 / 16
    ref = projection.DesignMap("sc", w.n, spacing=2, radius=r, octant=True)
    rng = np.random.default_rng(1616)
    x0 = rng.uniform(0.2, 0.8, ref.nvars)
    beta = 4.0
    rho = ref.forward(x0, beta)
    P = mixed.build(w.lattice, w.n, w.M, rho, w.phase1, w.phase0, w.penal)
    lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
    ctol = B.PC_CLUSTER_TOL_FP64 if precision == "fp64" else B.PC_CLUSTER_TOL_MIXED
    res = ogap.gap(lam, 6, rel_tol=ctol)
    g_ref = ref.backward(x0, beta, sensitivity.weighted(P, sols, res.weights))

    dm = DesignMap("sc", w.n, spacing=2, radius=r, octant=True)
    s = BandSolver.from_workload(w, precision=precision)
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    G = gap(ProjectFn.apply(x, dm, beta), s, 6)
    G.backward()
    tol_w, tol_g = (1e-9, 1e-5) if precision == "fp64" else (1e-6, 1e-4)
    assert abs(G.item() - res.gap) <= 4 * tol_w * abs(res.gap)
    rel = np.linalg.norm(x.grad.cpu().numpy() - g_ref) / np.linalg.norm(g_ref)
    assert rel <= tol_g, rel
    assert s.stats().status == B.PC_OK
    s.close()
    dm.close()


def test_design_loop_with_continuation_matches_oracle_loop(B):
    """maximize_gap on the free variables of an octant-symmetric reduced field (SC 8^3, M = 1,
    smooth gap(3,4)), beta 1, 1, 2, 2 over four MMA steps, against the oracle's loop."""
    from oracle import mma
    from paper_1603_06855_gb300.solver import BandSolver, DesignMap, heaviside_schedule, maximize_gap
    w = wl.sc8_binary_cube()
    r = 2.5 / 8
    ref = projection.DesignMap("sc", w.n, spacing=2, radius=r, octant=True)
    x0 = np.random.default_rng(88).uniform(0.3, 0.7, ref.nvars)
    kb = 50.0
    wref = 2 * np.pi * np.sqrt(w.phase1["E"] / w.phase1["rho"])
    s = BandSolver.from_workload(w, precision="fp64")
    dm = DesignMap("sc", w.n, spacing=2, radius=r, octant=True)
    x, hist = maximize_gap(s, torch.from_numpy(x0).cuda(), 3, kb, 4, design=dm, beta_every=2)
    assert s.stats().status == B.PC_OK
    xr, st, href = x0.copy(), mma.MMAState(), []
    for step in range(5):
        hb = heaviside_schedule(step, 2)
        rho = ref.forward(xr, hb)
        P = mixed.build(w.lattice, w.n, w.M, rho, w.phase1, w.phase0, w.penal)
        lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
        res = ogap.ks_gap(lam, 3, kb, omega_ref=wref)
        href.append(res.gap)
        if step < 4:
            xr = mma.step(xr, ref.backward(xr, hb, sensitivity.weighted(P, sols, res.weights)), st)
    assert np.allclose(hist, href, rtol=5e-6, atol=0), (hist, href)
    assert np.abs(x.cpu().numpy() - xr).max() <= 1e-3
    s.close()
    dm.close()
