"""GPU parity of the design update (pc_mma_step) and of the optimization loop built on it.

* k_mma_step against the oracle's MMA step, every step started from the same state (copied
  back from the device), 100003 variables (many blocks and a ragged tail), bounds [0, 1] and a
  shifted box.  Tolerance 1e-12 of the box: the device may fuse multiply-adds, which moves
  results by a few ulps; the history arrays are copies and must match exactly.
* maximize_gap (band structure, smooth gap, adjoint, MMA update, three times) on the SC 8^3 cube
  cell against the same loop run with the oracle's bands, gradient and MMA step, and the gap
  rising at every step.  The FP64 gradient is held to 1e-5 relative L2 of the oracle's by the
  parity tests; on the oracle's own loop a gradient perturbed by that much moved the gap history
  by at most 1.6e-6 relative and the design by 3.6e-4 (variables whose gradient is near the
  method's 1e-5 regulariser move most), so the history is allowed 5e-6 and the design 1e-3.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import gap as og
from oracle import mixed, mma, sensitivity

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


@pytest.mark.parametrize("xmin,xmax", [(0.0, 1.0), (-0.5, 2.0)])
def test_mma_step_matches_oracle(B, xmin, xmax):
    from paper_1603_06855_gb300.solver import MMA
    rng = np.random.default_rng(92)
    n = 100003
    span = xmax - xmin
    c = rng.uniform(xmin - 0.3 * span, xmax + 0.3 * span, n)
    x0 = rng.uniform(xmin, xmax, n)
    x0[:64] = xmin
    x0[64:128] = xmax
    x = torch.from_numpy(x0).cuda()
    opt = MMA(n, xmin, xmax)
    for it in range(12):
        xh = x.cpu().numpy()
        df = -2.0 * (xh - c) * (1.0 + rng.uniform(0, 1, n))
        h1, h2 = opt.xold1.cpu().numpy(), opt.xold2.cpu().numpy()
        lo, up = opt.low.cpu().numpy(), opt.upp.cpu().numpy()
        st = mma.MMAState(it=it, x1=None if it == 0 else h1, x2=None if it < 2 else h2,
                          L=None if it == 0 else lo, U=None if it == 0 else up)
        ref = mma.step(xh, df, st, xmin, xmax)
        opt.step(x, torch.from_numpy(df).cuda())
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * span, it
        assert np.abs(opt.low.cpu().numpy() - st.L).max() <= 1e-12 * span
        assert np.abs(opt.upp.cpu().numpy() - st.U).max() <= 1e-12 * span
        assert np.array_equal(opt.xold1.cpu().numpy(), xh)
        if it >= 1:
            assert np.array_equal(opt.xold2.cpu().numpy(), h1)
        assert np.all((got >= xmin) & (got <= xmax))
        x = torch.from_numpy(ref).cuda()   # continue both from the oracle's iterate
        opt.xold1.copy_(torch.from_numpy(xh))
        opt.low.copy_(torch.from_numpy(st.L))
        opt.upp.copy_(torch.from_numpy(st.U))
        if it >= 1:
            opt.xold2.copy_(torch.from_numpy(h1))


def test_maximize_gap_matches_oracle_loop(B):
    from paper_1603_06855_gb300.solver import BandSolver, maximize_gap
    w = wl.sc8_binary_cube()
    rng = np.random.default_rng(84)
    rho0 = np.clip(0.2 + 0.6 * w.rho + 0.05 * rng.standard_normal(w.n), 0.0, 1.0)
    beta = 50.0
    wref = 2 * np.pi * np.sqrt(w.phase1["E"] / w.phase1["rho"])

    s = BandSolver.from_workload(w, precision="fp64")
    x, hist = maximize_gap(s, torch.from_numpy(rho0).cuda(), 3, beta, 3)
    st = s.stats()
    assert st.status == B.PC_OK, B.pc_strerror(st.status)
    s.close()

    r = rho0.ravel().copy()
    ost = mma.MMAState()
    ref = []
    for step in range(4):
        P = mixed.build(w.lattice, w.n, w.M, r.reshape(w.n), w.phase1, w.phase0, w.penal)
        lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
        res = og.ks_gap(lam, 3, beta, omega_ref=wref)
        ref.append(res.gap)
        if step < 3:
            r = mma.step(r, sensitivity.weighted(P, sols, res.weights), ost)
    assert np.allclose(hist, ref, rtol=5e-6, atol=0), (hist, ref)
    assert all(b > a for a, b in zip(hist, hist[1:])), hist
    assert np.abs(x.cpu().numpy().ravel() - r).max() <= 1e-3
