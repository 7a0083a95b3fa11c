"""Uneven batch: 12 SC, 10 BCC and 10 FCC designs with N in {125, 343, 729, 1331} plane waves
and grids from 16^3 to 40^3, 48 k-points and 20 bands each, mixed form, evaluated in one call of
the batch interface (pc_batch_*: a work queue of the designs, largest first, drained by
concurrent workers).

* every design finishes with PC_OK and ascending, finite frequencies;
* one design per (lattice, N) bucket, the one with the smallest voxel grid (the dense oracle's
  element sums grow with the grid; the library's path does not change with it), is checked
  against the FP64 oracle at two sampled k-points: 1e-6 relative, |w - w_ref| / max(w_ref, 0.05
  max w_ref).  The oracle needs about 20 s per sampled k at N = 1331;
* the batch's bands and gap(6,7) gradients equal those of the same designs solved one context at
  a time (the same computation on other streams: 1e-12);
* the autotuner times its candidates on a small batch and records the fastest.
"""
import json

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


def _single(B, w):
    from paper_1603_06855_gb300.solver import BandSolver
    s = BandSolver(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.Q, w.penal, B.PC_MIXED, w.a)
    s.set_design(torch.from_numpy(w.rho.ravel()).cuda())
    om = s.bands().cpu().numpy()
    _, g = s.gap_and_grad(6)
    g = g.cpu().numpy()
    s.close()
    return om, g


def _err(got, ref):
    return np.max(np.abs(got - ref) / np.maximum(ref, 0.05 * ref.max()))


def test_uneven_batch32_one_call(B):
    from paper_1603_06855_gb300.solver import BatchSolver
    designs = wl.batch32_mixed()
    bs = BatchSolver(designs, B.PC_MIXED, workers=4)
    bs.set_designs([w.rho for w in designs])
    oms = [o.cpu().numpy() for o in bs.bands()]
    gaps, grads = bs.gap_and_grad(n_lower=[6] * len(designs))
    torch.cuda.synchronize()
    for d, w in enumerate(designs):
        st = bs.stats(d)
        assert st.status == B.PC_OK, (w.name, B.pc_strerror(st.status))
        assert np.all(np.isfinite(oms[d])) and np.all(np.diff(oms[d], axis=1) >= 0), w.name
    pick = {}
    for i, w in enumerate(designs):
        key = (w.lattice, (2 * w.M + 1) ** 3)
        if key not in pick or np.prod(w.n) < np.prod(designs[pick[key]].n):
            pick[key] = i
    assert len(pick) == 12, pick
    worst = {}
    for i in pick.values():
        w = designs[i]
        P = mixed.from_workload(w)
        ref = mixed.omega(mixed.bands(P, w.Q[SAMPLE_K], w.nbands))
        worst[w.name] = _err(oms[i][SAMPLE_K], ref)
    bad = {k: v for k, v in worst.items() if not v <= 1e-6}
    assert not bad, bad
    # the same designs one context at a time
    for i in (pick[("fcc", 729)], pick[("sc", 125)]):
        om1, g1 = _single(B, designs[i])
        assert np.abs(om1 - oms[i]).max() <= 1e-12 * om1.max()
        g = grads[i].cpu().numpy()
        assert np.linalg.norm(g - g1) <= 1e-12 * np.linalg.norm(g1)
    bs.close()


def test_autotuner_records_a_measured_choice(B, tmp_path):
    from paper_1603_06855_gb300 import autotune
    designs = [w for w in wl.batch32_mixed() if (2 * w.M + 1) ** 3 <= 343][:6]
    path = str(tmp_path / "autotune.json")
    props = torch.cuda.get_device_properties(0)
    cands = ((1, 0), (3, 0), (3, 1))
    w, g = autotune.choose(designs, B.PC_MIXED, [d.rho for d in designs], autotune.measure_batch, props.name,
                           props.multi_processor_count, path, candidates=cands)
    rec = json.load(open(path))
    (entry,) = rec.values()
    assert [w, g] == entry["choice"] and set(entry["seconds"]) == {"1,0", "3,0", "3,1"}
    assert all(t > 0 for t in entry["seconds"].values())
    assert entry["seconds"][f"{w},{g}"] == min(entry["seconds"].values())
