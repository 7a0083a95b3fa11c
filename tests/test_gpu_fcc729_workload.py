"""Parity on the benchmark workload itself, in the benchmark's launch configuration.

FCC cell, 32^3 voxels, M = 4 (N = 729 plane waves), 100 k-points along the high-symmetry path,
20 bands, in both forms: the library solves all 100 k-points at once (the mixed form, with this
many k-points, as concurrent k groups on separate streams: the configuration the bench times;
the FP64 form, the bench's plain FP64 GPU form, on one stream).  The oracle solves a sample of
k-points taken from different groups; on that sample:

* eigenfrequencies within 1e-6 (mixed) and 1e-9 (FP64) relative (|w - w_ref| / max(w_ref,
  0.05 max w_ref); the Gamma zero modes on lambda, |lambda| <= 1e-9 lambda_max);
* the adjoint gradient of a seeded weighted sum of the sampled eigenvalues (every band at the
  sampled k-points, the Gamma zero modes excluded, zero weight elsewhere) within 1e-4 (mixed) and
  1e-5 (FP64) relative L2, and the weighted sum itself within the frequency tolerance.
"""
import functools

import numpy as np
import pytest

import workloads as wl
from oracle import mixed, sensitivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE = [0, 23, 50, 77, 99]  # Gamma, both halves of the path, the last point
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
def oracle_sample():
    w = wl.fcc32_levelset()
    P = mixed.from_workload(w)
    lam_ref, sols = mixed.bands(P, w.Q[SAMPLE], w.nbands, keep=True)
    return w, P, lam_ref, sols


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fcc729_bench_workload_sampled_k(B, precision):
    from paper_1603_06855_gb300.solver import BandSolver
    w, P, lam_ref, sols = oracle_sample()
    prec = B.PC_MIXED if precision == "mixed" else B.PC_FP64
    s = BandSolver.from_workload(w, precision=prec, device=torch.device("cuda", 0))
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    om = s.bands().cpu().numpy()
    st = s.stats()
    assert st.status == B.PC_OK, B.pc_strerror(st.status)

    lmax = lam_ref.max()
    ref = np.sqrt(np.maximum(lam_ref, 0.0))
    zero = np.abs(lam_ref) <= 1e-9 * lmax
    got = om[SAMPLE]
    err = np.abs(got - ref) / np.maximum(ref, 0.05 * ref.max())
    assert err[~zero].max() <= TOL_W[precision], err[~zero].max()
    assert np.all(got[zero] ** 2 <= 1e-9 * lmax)

    rng = np.random.default_rng(2187)
    wts_s = rng.uniform(0.5, 1.5, size=lam_ref.shape) / lmax
    wts_s[zero] = 0.0
    wts = np.zeros((w.nk, w.nbands))
    wts[SAMPLE] = wts_s
    g_ref = sensitivity.weighted(P, sols, wts_s)
    val, grad = s.gap_and_grad(mode=B.PC_GRAD_ALLBANDS, weights=torch.from_numpy(wts))
    assert abs(val.cpu().numpy()[0] - np.sum(wts_s * lam_ref)) <= 2 * TOL_W[precision] * np.sum(np.abs(wts_s * lam_ref))
    rel = np.linalg.norm(grad.cpu().numpy().ravel() - g_ref) / np.linalg.norm(g_ref)
    assert rel <= TOL_G[precision], rel
    s.close()
