"""Uneven batch: 12 SC, 10 BCC and 10 FCC designs with N in {125, 343, 729, 1331} plane waves
and grids from 16^3 to 40^3, 48 k-points and 20 bands each, mixed form.

Every design runs through the library (all 48 k-points: with this many the block iteration
runs as concurrent k groups); each must finish with PC_OK and ascending, finite frequencies.
One design per (lattice, N) bucket, the one with the smallest voxel grid (the dense oracle's
element sums grow with the grid; the library's path does not change with it), is checked
against the FP64 oracle at two sampled k-points.  Tolerance: 1e-6 relative,
|w - w_ref| / max(w_ref, 0.05 max w_ref).  The oracle needs about 20 s per sampled k at
N = 1331 (7986 x 7986 compliance block).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import mixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE_K = [5, 30]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


def _run(B, w, precision, Q=None):
    from paper_1603_06855_gb300.solver import BandSolver
    s = BandSolver(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.Q if Q is None else Q, w.penal, precision,
                   w.a)
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    om = s.bands().cpu().numpy()
    st = s.stats()
    s.close()
    return om, st


def _err(got, ref):
    return np.max(np.abs(got - ref) / np.maximum(ref, 0.05 * ref.max()))


def test_uneven_batch32(B):
    designs = wl.batch32_mixed()
    pick = {}
    for i, w in enumerate(designs):
        key = (w.lattice, (2 * w.M + 1) ** 3)
        if key not in pick or np.prod(w.n) < np.prod(designs[pick[key]].n):
            pick[key] = i
    assert len(pick) == 12, pick
    checked = set(pick.values())
    worst = {}
    for i, w in enumerate(designs):
        om, st = _run(B, w, B.PC_MIXED)
        assert st.status == B.PC_OK, (w.name, B.pc_strerror(st.status))
        assert np.all(np.isfinite(om)) and np.all(np.diff(om, axis=1) >= 0), w.name
        if i not in checked:
            continue
        P = mixed.from_workload(w)
        ref = mixed.omega(mixed.bands(P, w.Q[SAMPLE_K], w.nbands))
        worst[w.name] = _err(om[SAMPLE_K], ref)
    assert len(worst) == 12, worst
    bad = {k: v for k, v in worst.items() if not v <= 1e-6}
    assert not bad, bad
