"""GPU parity of the variants of the path (beyond the paper's defaults), through the C ABI:

* eq. combinematerial read literally (PC_LAW_YOUNG: Young's modulus and Poisson's ratio linear in
  chi, every element the isotropic material they give; Methods, "Topology optimization
  formulation"): the compliance Toeplitz operators against the oracle's element sums (1e-12), the
  bands (1e-9 FP64 / 1e-6 mixed) and the gap(6,7) gradient (1e-5 / 1e-4 relative L2), whose
  adjoint now carries a per-element d(compliance)/d(chi);
* the warm start across designs: a second, nearby design started from the first one's final Ritz
  block needs fewer block iterations and gives the oracle's bands and gradient; a block exported
  from one context and imported into another reproduces the warm-started result.
"""
import functools

import numpy as np
import pytest

import workloads as wl
from oracle import gap as ogap
from oracle import mixed, sensitivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = {"fp64": 1e-9, "mixed": 1e-6}
TOL_G = {"fp64": 1e-5, "mixed": 1e-4}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


@functools.lru_cache(maxsize=None)
def young_oracle():
    w = wl.sc16_grf()
    P = mixed.build(w.lattice, w.n, w.M, w.rho, w.phase1, w.phase0, w.penal, law="young")
    lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
    return w, P, lam, sols


def omega_err(om, lam_ref):
    ref = mixed.omega(lam_ref)
    zero = np.abs(lam_ref) <= 1e-9 * lam_ref.max()
    assert np.all(om[zero] ** 2 <= 1e-9 * lam_ref.max())
    return np.max(np.where(zero, 0.0, np.abs(om - ref) / np.maximum(ref, 0.05 * ref.max())))


def test_young_law_assembly(B):
    from paper_1603_06855_gb300.solver import BandSolver
    w, P, _, _ = young_oracle()
    s = BandSolver.from_workload(w, precision="fp64", law="young")
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    torch.cuda.synchronize()
    N = P.N
    T = s.export(B.PC_EXPORT_TOEP).view(np.complex128).reshape(3, N, N)
    Tf1 = P.Phi[:N, :N] + 2 * P.Phi[:N, N:2 * N]       # D11 + 2 D12 = (1 - 2 nu) / E per element
    Tf2 = 0.5 * P.Phi[3 * N:4 * N, 3 * N:4 * N]        # D44 / 2 = (1 + nu) / E per element
    for got, ref in ((T[0], P.Omega[:N, :N]), (T[1], Tf1), (T[2], Tf2)):
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_young_law_bands_and_gradient(B, precision):
    from paper_1603_06855_gb300.solver import BandSolver
    w, P, lam, sols = young_oracle()
    s = BandSolver.from_workload(w, precision=precision, law="young")
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    om = s.bands().cpu().numpy()
    assert omega_err(om, lam) <= TOL_W[precision]
    ctol = B.PC_CLUSTER_TOL_FP64 if precision == "fp64" else B.PC_CLUSTER_TOL_MIXED
    r = ogap.gap(lam, 6, rel_tol=ctol)
    g_ref = sensitivity.weighted(P, sols, r.weights)
    gap, grad = s.gap_and_grad(6)
    assert abs(gap.item() - r.gap) <= 4 * TOL_W[precision] * abs(r.gap)
    rel = np.linalg.norm(grad.cpu().numpy().ravel() - g_ref) / np.linalg.norm(g_ref)
    assert rel <= TOL_G[precision], rel
    assert s.stats().status == B.PC_OK
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_and_block_transfer(B, precision):
    from paper_1603_06855_gb300.solver import BandSolver
    w = wl.sc16_grf()
    rng = np.random.default_rng(2718)
    rho_b = np.clip(w.rho + 0.02 * rng.standard_normal(w.n), 0.0, 1.0)
    P = mixed.build(w.lattice, w.n, w.M, rho_b, w.phase1, w.phase0, w.penal)
    lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
    ctol = B.PC_CLUSTER_TOL_FP64 if precision == "fp64" else B.PC_CLUSTER_TOL_MIXED
    r = ogap.gap(lam, 6, rel_tol=ctol)
    g_ref = sensitivity.weighted(P, sols, r.weights)

    cold = BandSolver.from_workload(w, precision=precision)
    cold.set_design(torch.from_numpy(rho_b.ravel()).cuda())
    cold.bands()
    it_cold = cold.stats().iterations
    cold.close()

    s = BandSolver.from_workload(w, precision=precision)
    s.set_warm_start(True)
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    s.bands()
    block_a = s.export(B.PC_EXPORT_BLOCK)
    s.set_design(torch.from_numpy(rho_b.ravel()).cuda())
    om = s.bands().cpu().numpy()
    st = s.stats()
    assert st.status == B.PC_OK
    assert st.iterations < it_cold, (st.iterations, it_cold)
    assert omega_err(om, lam) <= TOL_W[precision]
    _, grad = s.gap_and_grad(6)
    rel = np.linalg.norm(grad.cpu().numpy().ravel() - g_ref) / np.linalg.norm(g_ref)
    assert rel <= TOL_G[precision], rel

    t = BandSolver.from_workload(w, precision=precision)
    t.import_block(block_a)
    t.set_design(torch.from_numpy(rho_b.ravel()).cuda())
    om2 = t.bands().cpu().numpy()
    assert t.stats().iterations == st.iterations
    assert np.abs(om2 - om).max() <= 1e-12 * om.max()
    s.close()
    t.close()
