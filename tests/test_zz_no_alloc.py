"""The allocation-free entry point against the regular path.

pc_structure_factors_noalloc serves callers that may not allocate device memory while they
run; it works in a fixed device array instead of context workspaces.  This file is collected
last so that a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


def _regular(B, w, rho):
    from paper_1603_06855_gb300.solver import BandSolver
    s = BandSolver(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.Q, w.penal, B.PC_FP64, w.a)
    s.set_design(torch.from_numpy(rho.ravel()).cuda())
    torch.cuda.synchronize()
    out = s.export(B.PC_EXPORT_SFAC)
    s.close()
    return out


def test_noalloc_matches_regular_path_twice(B):
    """Two calls in a row (different designs and sizes) against pc_set_design's structure factors."""
    cases = [wl.sc16_grf(), wl.sc8_binary_cube()]
    cases[1].rho = np.clip(0.2 + 0.6 * cases[1].rho + 0.05 * np.random.default_rng(3).standard_normal(cases[1].n), 0, 1)
    stream = torch.cuda.current_stream().cuda_stream
    for w in cases:
        ref = _regular(B, w, w.rho)
        p = B.make_params(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.penal)
        rho = torch.from_numpy(w.rho.ravel()).cuda()
        L = 4 * w.M + 1
        out = torch.full((3 * L ** 3 * 2,), float("nan"), dtype=torch.float64, device="cuda")
        assert B.pc_structure_factors_noalloc(p, rho.data_ptr(), out.data_ptr(), stream) == B.PC_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_rejects_oversized_grids(B):
    w = wl.sc16_grf()
    p = B.make_params(w.lattice, (48, 48, 48), w.M, w.nbands, w.phase1, w.phase0, w.penal)
    rho = torch.zeros(48 ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros(3 * (4 * w.M + 1) ** 3 * 2, dtype=torch.float64, device="cuda")
    assert B.pc_structure_factors_noalloc(p, rho.data_ptr(), out.data_ptr(), 0) == B.PC_ETOOBIG
