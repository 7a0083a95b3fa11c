"""GPU band structure of the paper's sphere-inclusion cells, through the C ABI.

Tungsten-carbide spheres in epoxy with the constants of the paper's volume-fraction scans (Results,
note on normalized band gaps), one sphere per primitive cell at the volume fraction where each
scan peaks, M = 3 on 24^3 voxels, sampled at the distinct high-symmetry points.  Checked:

* frequencies against the FP64 oracle: 1e-9 (FP64 form) and 1e-6 (mixed form), floored relative
  error as in the other parity tests; Gamma zero modes on lambda;
* gap(6,7) against the oracle's gap: |dG| <= 2 tol for frequencies within relative tol, so
  3 tol is allowed;
* the adjoint gradient of gap(6,7) against the oracle's: relative L2 1e-5 (FP64) and 1e-4
  (mixed), with the cluster window of each form on both sides;
* the printed maxima within 3 percentage points, the approximate pin the oracle carries (the
  paper states neither the cutoff nor the grid of these scans).

The cells have the full cubic symmetry, so many bands are degenerate at the high-symmetry
points; the edges of gap(6,7) are not (the nearest band is 1-17 % away at the extremal
k-points).  Degenerate edges are covered by tests/test_gpu_degenerate_clusters.py.
"""
import functools
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import gap as ogap
from oracle import mixed, sensitivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = {"fp64": 1e-9, "mixed": 1e-6}
TOL_G = {"fp64": 1e-5, "mixed": 1e-4}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sphere_inclusions.json")
CASES = {c["lattice"]: c for c in json.load(open(GOLDEN))["cases"]}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


@functools.lru_cache(maxsize=None)
def sphere_workload(lattice):
    n = (24, 24, 24)
    c = CASES[lattice]
    rho = wl.sphere_inclusion(lattice, n, c["volume_fraction"])
    return wl.Workload(f"{lattice}24_M3_sphere", lattice, n, 3, 8, wl.high_symmetry_points(lattice),
                       rho, 1.0, (6,), 0, 1.0, dict(wl.PAPER_WC), dict(wl.PAPER_EPOXY))


@functools.lru_cache(maxsize=None)
def oracle_bands(lattice):
    w = sphere_workload(lattice)
    P = mixed.from_workload(w)
    lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
    return P, lam, sols


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lattice", ["sc", "bcc", "fcc"])
def test_sphere_inclusion_bands_and_gap(B, lattice, precision):
    from paper_1603_06855_gb300.solver import BandSolver
    w = sphere_workload(lattice)
    P, lam_ref, sols = oracle_bands(lattice)
    ref = mixed.omega(lam_ref)
    s = BandSolver(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.Q, w.penal, precision, w.a)
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    om = s.bands().cpu().numpy()
    g, grad = s.gap_and_grad(6, B.PC_GAP_OMEGA)
    g = float(g.cpu().item())
    st = s.stats()
    assert st.status == B.PC_OK, B.pc_strerror(st.status)
    floor = 0.05 * ref.max()
    zero = np.abs(lam_ref) <= 1e-9 * lam_ref.max()
    assert np.all(om[zero] ** 2 <= 1e-9 * lam_ref.max()), "zero modes"
    err = np.max(np.where(zero, 0.0, np.abs(om - ref) / np.maximum(ref, floor)))
    assert err <= TOL_W[precision], (err, st.iterations, st.max_residual)
    ctol = B.PC_CLUSTER_TOL_FP64 if precision == "fp64" else B.PC_CLUSTER_TOL_MIXED
    r = ogap.gap(lam_ref, 6, rel_tol=ctol)
    g_ref = r.gap
    assert abs(g - g_ref) <= 3 * TOL_W[precision], (g, g_ref)
    gr_ref = sensitivity.weighted(P, sols, r.weights)
    rel = np.linalg.norm(grad.cpu().numpy().ravel() - gr_ref) / np.linalg.norm(gr_ref)
    assert rel <= TOL_G[precision], rel
    assert abs(100 * g - CASES[lattice]["printed_gap_pct"]) <= 3.0, (g, CASES[lattice])
    s.close()
