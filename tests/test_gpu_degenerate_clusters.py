"""Adjoint gradients at degenerate band clusters, through the C ABI, against the oracle.

Tungsten-carbide sphere in epoxy (the paper's constants and its SC scan optimum, volume fraction
0.412; Results, note on normalized band gaps) on 16^3 voxels with M = 2, at the four
high-symmetry points Gamma, X, M, R of the simple cubic zone.  The cell has the full cubic
symmetry, so the bands come in exact multiplets at Gamma, X and R.  Two objectives put the
extremal (k, band) of the gap inside such a multiplet:

* gap(7, 8): band 7 peaks at R inside the doublet {7, 8}, band 8 bottoms at X inside {7, 8};
* gap(10, 11): band 10 peaks at Gamma inside the triplet {10, 11, 12}.

Neither eigenvalue of a multiplet is differentiable on its own; the library hands the weight of
the extremal band to every band of its cluster in equal shares (the gradient of the cluster-mean
eigenvalue, Methods, eqs. sensitivityew, diffOmega, diffPhi), which does not depend on the
basis the eigensolver picked inside the cluster.  Checked, in both forms:

* the gap against the oracle's (same cluster window, PC_CLUSTER_TOL_*), the weight pattern, and
  the gradient against the oracle's cluster-mean gradient: relative L2 1e-5 (FP64) and 1e-4
  (mixed);
* the gradient is invariant under the exact symmetries of the discrete problem at both extremal
  wavevectors: inversion through the sphere centre (with time reversal it maps every k-point's
  plane-wave set onto itself) and the x <-> z swap (it fixes X = (0, 1/2, 0), R and Gamma).
  The gradient of one arbitrary member of the R doublet differs from its x <-> z image by 50 %
  (oracle); mirrors of single axes are not exact symmetries, since they move R to an equivalent
  point with a different truncated plane-wave set.
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
VF_SC = {c["lattice"]: c for c in json.load(open(GOLDEN))["cases"]}["sc"]["volume_fraction"]
NBANDS = 14


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


@functools.lru_cache(maxsize=None)
def cell():
    n = (16, 16, 16)
    rho = wl.sphere_inclusion("sc", n, VF_SC)
    w = wl.Workload("sc16_M2_sphere", "sc", n, 2, NBANDS, wl.high_symmetry_points("sc"), rho, 1.0, (7, 10), 0, 1.0,
                    dict(wl.PAPER_WC), dict(wl.PAPER_EPOXY))
    P = mixed.from_workload(w)
    lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
    return w, P, lam, sols


def cluster_sizes(weights):
    return sorted(int(np.count_nonzero(row)) for row in weights if np.any(row))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_at_degenerate_clusters(B, precision):
    from paper_1603_06855_gb300.solver import BandSolver
    w, P, lam_ref, sols = cell()
    ctol = B.PC_CLUSTER_TOL_FP64 if precision == "fp64" else B.PC_CLUSTER_TOL_MIXED
    s = BandSolver.from_workload(w, precision=precision)
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    om = s.bands().cpu().numpy()
    st = s.stats()
    assert st.status == B.PC_OK, B.pc_strerror(st.status)
    ref = mixed.omega(lam_ref)
    zero = np.abs(lam_ref) <= 1e-9 * lam_ref.max()
    err = np.max(np.where(zero, 0.0, np.abs(om - ref) / np.maximum(ref, 0.05 * ref.max())))
    assert err <= TOL_W[precision], err
    for n_lower, sizes in ((7, [2, 2]), (10, [1, 3])):
        r = ogap.gap(lam_ref, n_lower, rel_tol=ctol)
        # the objective does sit on exact multiplets of the oracle
        assert cluster_sizes(r.weights) == sizes, (n_lower, r.weights)
        g_ref = sensitivity.weighted(P, sols, r.weights)
        gap, grad = s.gap_and_grad(n_lower)
        assert abs(gap.item() - r.gap) <= 4 * TOL_W[precision] * abs(r.gap), (gap.item(), r.gap)
        wts = s.export(B.PC_EXPORT_WEIGHT).reshape(w.nk, w.nbands)
        assert np.array_equal(np.nonzero(wts), np.nonzero(r.weights)), (n_lower, wts, r.weights)
        assert np.allclose(wts, r.weights, rtol=1e-5, atol=0.0)
        g = grad.cpu().numpy()
        rel = np.linalg.norm(g.ravel() - g_ref) / np.linalg.norm(g_ref)
        assert rel <= TOL_G[precision], (n_lower, rel)
        # symmetries shared by the design and both extremal wavevectors
        for image in (g[::-1, ::-1, ::-1], np.transpose(g, (2, 1, 0))):
            d = np.linalg.norm(image - g) / np.linalg.norm(g)
            assert d <= TOL_G[precision], (n_lower, d)
    s.close()
