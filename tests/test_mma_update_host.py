"""The per-variable update that k_mma_step runs (csrc/mma_update.cuh), compiled for the host,
against the oracle's MMA step, step by step on seeded data (CPU only).

The host build has no fused multiply-adds (-ffp-contract=off), like the oracle, so the two
agree to rounding; every step starts both from the same state, so the branch on the
oscillation sign sees the same inputs.  The device build may fuse multiply-adds; its parity
test on the GPU allows for that."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import gap as og
from oracle import mixed, mma, sensitivity

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1603_06855_gb300", "csrc")

HARNESS = r"""
#include "mma_update.cuh"
extern "C" void mma_host(long long n, double* x, const double* df, double* xo1, double* xo2, double* low,
                         double* upp, int iter, double xmin, double xmax) {
  for (long long i = 0; i < n; ++i) {
    double xn;
    mma_box_update(x[i], df[i], iter, xmin, xmax, xo1 + i, xo2 + i, low + i, upp + i, &xn);
    x[i] = xn;
  }
}
"""


@pytest.fixture(scope="module")
def host_update(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("mma_host")
    src, lib = d / "harness.cpp", d / "libmma_host.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(lib)],
                   check=True, capture_output=True)
    so = ctypes.CDLL(str(lib))
    P = ctypes.c_void_p
    so.mma_host.argtypes = [ctypes.c_longlong, P, P, P, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    so.mma_host.restype = None

    def run(x, df, x1, x2, lo, up, it, xmin, xmax):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in (x, df, x1, x2, lo, up)]
        so.mma_host(len(arrs[0]), *[a.ctypes.data for a in arrs], it, xmin, xmax)
        x, _, x1, x2, lo, up = arrs
        return x, x1, x2, lo, up
    run.raw = so.mma_host   # same argument order as pc_mma_step, without the stream
    return run


@pytest.mark.parametrize("xmin,xmax", [(0.0, 1.0), (-0.5, 2.0)])
def test_update_matches_oracle_step_by_step(host_update, xmin, xmax):
    rng = np.random.default_rng(91)
    n = 257
    c = rng.uniform(xmin - 0.3 * (xmax - xmin), xmax + 0.3 * (xmax - xmin), n)
    x = rng.uniform(xmin, xmax, n)
    x[:8] = xmin          # start on the bounds, too
    x[8:16] = xmax
    st = mma.MMAState()
    h1 = h2 = lo = up = np.zeros(n)
    for it in range(30):
        df = -2.0 * (x - c) * (1.0 + rng.uniform(0, 1, n))   # a non-quadratic ascent direction
        hx, h1n, h2n, lon, upn = host_update(x, df, h1, h2, lo, up, it, xmin, xmax)
        # the oracle from the same state
        ost = mma.MMAState(it=it, x1=None if it == 0 else h1.copy(), x2=None if it < 2 else h2.copy(),
                           L=None if it == 0 else lo.copy(), U=None if it == 0 else up.copy())
        ox = mma.step(x, df, ost, xmin, xmax)
        assert np.abs(hx - ox).max() <= 1e-13 * (xmax - xmin), it
        assert np.abs(lon - ost.L).max() <= 1e-13 * (xmax - xmin) and np.abs(upn - ost.U).max() <= 1e-13 * (xmax - xmin)
        assert np.array_equal(h1n, x)
        if it >= 1:
            assert np.array_equal(h2n, h1)
        assert np.all((hx >= xmin) & (hx <= xmax))
        x, h1, h2, lo, up = hx, h1n, h2n, lon, upn


def test_binding_wrapper_reports_errors():
    from paper_1603_06855_gb300 import binding as B, build_lib
    if not os.path.exists(B.LIB_PATH):
        build_lib.build()
    with pytest.raises(B.PhononicError):
        B.pc_mma_step(0, 0, 0, 0, 0, 0, 0, 0)


@pytest.fixture
def cpu_solver_layer(host_update, monkeypatch):
    """solver.MMA and solver.maximize_gap on CPU tensors: pc_mma_step replaced by the host build
    of the kernel's update (same argument order), the CUDA stream by a null handle."""
    import types
    from paper_1603_06855_gb300 import solver as S

    def fake_step(n, x, df, x1, x2, lo, up, it, xmin, xmax, stream):
        assert stream == 0
        host_update.raw(n, x, df, x1, x2, lo, up, it, xmin, xmax)
    monkeypatch.setattr(S.B, "pc_mma_step", fake_step)
    monkeypatch.setattr(S.torch.cuda, "current_stream", lambda device=None: types.SimpleNamespace(cuda_stream=0))
    return S


def test_mma_layer_matches_oracle(cpu_solver_layer):
    S = cpu_solver_layer
    rng = np.random.default_rng(93)
    n = 300
    c = rng.uniform(-0.3, 1.3, n)
    x = torch.from_numpy(rng.uniform(0, 1, n))
    opt = S.MMA(n, device="cpu")
    ref, st = x.numpy().copy(), mma.MMAState()
    for it in range(15):
        df = -2.0 * (ref - c)
        opt.step(x, torch.from_numpy(df))
        ref = mma.step(ref, df, st)
        assert np.abs(x.numpy() - ref).max() <= 1e-13, it
    assert opt.iteration == 15
    with pytest.raises(ValueError):
        opt.step(x[:10], torch.zeros(10, dtype=torch.float64))


def test_maximize_gap_loop_matches_oracle_loop(cpu_solver_layer):
    S = cpu_solver_layer
    w = wl.sc8_binary_cube()
    rng = np.random.default_rng(84)
    rho0 = np.clip(0.2 + 0.6 * w.rho + 0.05 * rng.standard_normal(w.n), 0.0, 1.0)
    beta = 50.0
    wref = 2 * np.pi * np.sqrt(w.phase1["E"] / w.phase1["rho"])

    def evaluate(r):
        P = mixed.build(w.lattice, w.n, w.M, r.reshape(w.n), w.phase1, w.phase0, w.penal)
        lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
        res = og.ks_gap(lam, 3, beta, omega_ref=wref)
        return res.gap, sensitivity.weighted(P, sols, res.weights)

    class OracleSolver:
        """The solver calls maximize_gap makes, answered by the oracle on CPU tensors."""
        device = torch.device("cpu")
        n = w.n

        def __init__(self):
            self.calls = []

        def set_design(self, rho):
            assert rho.numel() == w.rho.size and rho.dtype == torch.float64
            self.rho = rho.detach().numpy().copy()
            self.calls.append("set_design")

        def bands(self):
            self.calls.append("bands")

        def gap_ks_and_grad(self, n_lower, b, need_grad=True):
            assert (n_lower, b) == (3, beta)
            self.calls.append("gap")
            g, grad = evaluate(self.rho)
            return torch.tensor([g], dtype=torch.float64), torch.from_numpy(grad.reshape(w.n)) if need_grad else None

    sol = OracleSolver()
    rho_in = torch.from_numpy(rho0.copy())
    x, hist = S.maximize_gap(sol, rho_in, 3, beta, 3)
    assert sol.calls == ["set_design", "bands", "gap"] * 4
    r, st, ref = rho0.ravel().copy(), mma.MMAState(), []
    for step in range(4):
        g, grad = evaluate(r)
        ref.append(g)
        if step < 3:
            r = mma.step(r, grad, st)
    assert np.allclose(hist, ref, rtol=1e-12, atol=0)
    assert tuple(x.shape) == w.n and np.abs(x.numpy().ravel() - r).max() <= 1e-13
    assert np.array_equal(rho_in.numpy(), rho0)  # the caller's design is not modified in place


def test_heaviside_schedule():
    from paper_1603_06855_gb300.solver import heaviside_schedule
    assert [heaviside_schedule(s, 2) for s in range(8)] == [1, 1, 2, 2, 4, 4, 8, 8]
    assert heaviside_schedule(100, 1) == 64.0


def test_maximize_gap_through_design_map_matches_oracle_loop(cpu_solver_layer):
    """The loop on free design variables: every step projects them (reduced field, SC octant,
    beta from the continuation), evaluates the smooth gap on the densities and chains its gradient
    back through the map; the map and the solver are answered by the oracle on CPU tensors."""
    from oracle import projection
    S = cpu_solver_layer
    w = wl.sc8_binary_cube()
    dm = projection.DesignMap("sc", w.n, spacing=2, radius=2.5 / 8, octant=True)
    rng = np.random.default_rng(85)
    x0 = rng.uniform(0.3, 0.7, dm.nvars)
    beta = 50.0
    wref = 2 * np.pi * np.sqrt(w.phase1["E"] / w.phase1["rho"])

    def evaluate(r):
        P = mixed.build(w.lattice, w.n, w.M, r.reshape(w.n), w.phase1, w.phase0, w.penal)
        lam, sols = mixed.bands(P, w.Q, w.nbands, keep=True)
        res = og.ks_gap(lam, 3, beta, omega_ref=wref)
        return res.gap, sensitivity.weighted(P, sols, res.weights)

    class OracleSolver:
        device = torch.device("cpu")
        n = w.n

        def set_design(self, rho):
            self.rho = rho.detach().numpy().copy()

        def bands(self):
            pass

        def gap_ks_and_grad(self, n_lower, b, need_grad=True):
            g, grad = evaluate(self.rho)
            return torch.tensor([g], dtype=torch.float64), torch.from_numpy(grad.reshape(w.n)) if need_grad else None

    class OracleDesign:
        betas = []

        def project(self, x, hb):
            self.x, self.hb = x.numpy().copy(), hb
            self.betas.append(hb)
            return torch.from_numpy(dm.forward(self.x, hb))

        def backprop(self, g):
            return torch.from_numpy(dm.backward(self.x, self.hb, g.numpy()))

    des = OracleDesign()
    x, hist = S.maximize_gap(OracleSolver(), torch.from_numpy(x0.copy()), 3, beta, 4, design=des, beta_every=2)
    assert des.betas == [1.0, 1.0, 2.0, 2.0, 4.0]
    r, st, ref = x0.copy(), mma.MMAState(), []
    for step in range(5):
        hb = S.heaviside_schedule(step, 2)
        g, grad = evaluate(dm.forward(r, hb))
        ref.append(g)
        if step < 4:
            r = mma.step(r, dm.backward(r, hb, grad), st)
    assert np.allclose(hist, ref, rtol=1e-12, atol=0)
    assert x.shape == (dm.nvars,) and np.abs(x.numpy() - r).max() <= 1e-13
