"""Torch-facing wrapper: device memory and streams come from PyTorch, every computation
from libphononic.so.  ``GapFn`` maps a density field to the normalized gap objective
(Methods, eq. obj) with the adjoint gradient (Methods, eq. sensitivityew) as backward."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class BandSolver:
    """One design context: lattice, grid, cutoff, bands, precision and a k-point set."""

    def __init__(self, lattice, n, M, nbands, phase1, phase0, Q, penal=1.0, precision=B.PC_FP64, a=1.0,
                 tol=0.0, max_iter=0, device="cuda"):
        if isinstance(precision, str):
            precision = {"fp64": B.PC_FP64, "mixed": B.PC_MIXED}[precision]
        self.device = torch.device(device)
        self.n = tuple(int(x) for x in n)
        self.nbands = int(nbands)
        self.params = B.make_params(lattice, n, M, nbands, phase1, phase0, penal, precision, a, tol, max_iter)
        self.ctx = B.pc_create(self.params)
        self.Q = np.ascontiguousarray(Q, dtype=np.float64)
        B.pc_set_kpoints(self.ctx, self.Q)
        self.nk = self.Q.shape[0]
        self._rho = None

    @classmethod
    def from_workload(cls, w, precision=B.PC_FP64, **kw):
        return cls(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.Q, w.penal, precision, w.a, **kw)

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def set_design(self, rho: torch.Tensor) -> None:
        rho = rho.detach().to(self.device, torch.float64).contiguous()
        if rho.numel() != self.n[0] * self.n[1] * self.n[2]:
            raise ValueError("density size does not match the grid")
        self._rho = rho  # keeps the buffer alive while kernels read it
        B.pc_set_design(self.ctx, rho.data_ptr(), self._stream())

    def bands(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.nk, self.nbands), dtype=torch.float64, device=self.device)
        B.pc_bands(self.ctx, out.data_ptr(), self._stream())
        return out

    def gap_and_grad(self, n_lower: int = 1, mode: int = B.PC_GAP_OMEGA, weights: torch.Tensor | None = None,
                     need_grad: bool = True, gap_out=None, grad_out=None):
        gap = gap_out if gap_out is not None else torch.empty(1, dtype=torch.float64, device=self.device)
        grad = None
        if need_grad:
            grad = grad_out if grad_out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        wptr = 0
        if weights is not None:
            weights = weights.to(self.device, torch.float64).contiguous()
            wptr = weights.data_ptr()
        B.pc_gap_and_grad(self.ctx, n_lower, mode, wptr, gap.data_ptr(), grad.data_ptr() if grad is not None else 0,
                          self._stream())
        return gap, grad

    def gap_ks_and_grad(self, n_lower: int, beta: float, need_grad: bool = True):
        """Smooth (KS) omega-form gap between bands n_lower and n_lower + 1 and its gradient."""
        gap = torch.empty(1, dtype=torch.float64, device=self.device)
        grad = torch.empty(self.n, dtype=torch.float64, device=self.device) if need_grad else None
        B.pc_gap_ks_and_grad(self.ctx, n_lower, float(beta), gap.data_ptr(),
                             grad.data_ptr() if grad is not None else 0, self._stream())
        return gap, grad

    def apply_operator(self, k: int, x: torch.Tensor):
        """SI A(k) x and Omega x for x of shape (ncols, 3N) complex128 (FP64 operator path)."""
        x = x.to(self.device, torch.complex128).contiguous()
        ax = torch.empty_like(x)
        ox = torch.empty_like(x)
        B.pc_apply_operator(self.ctx, k, x.shape[0], x.data_ptr(), ax.data_ptr(), ox.data_ptr(), self._stream())
        return ax, ox

    def export(self, which: int) -> np.ndarray:
        return B.pc_export(self.ctx, which)

    def stats(self):
        return B.pc_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            B.pc_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GapFn(torch.autograd.Function):
    """rho (n0, n1, n2) float64 CUDA tensor -> normalized gap between bands n_lower and n_lower+1."""

    @staticmethod
    def forward(ctx, rho, solver: BandSolver, n_lower: int, mode: int = B.PC_GAP_OMEGA):
        solver.set_design(rho)
        solver.bands()
        gap, grad = solver.gap_and_grad(n_lower, mode, need_grad=True)
        ctx.save_for_backward(grad)
        return gap[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None


def gap(rho: torch.Tensor, solver: BandSolver, n_lower: int, mode: int = B.PC_GAP_OMEGA) -> torch.Tensor:
    return GapFn.apply(rho, solver, n_lower, mode)


class MMA:
    """Device state of the design update of eq. topopt (method of moving asymptotes with the
    bounds as the only constraint) for n variables; each step is one pc_mma_step launch."""

    def __init__(self, n: int, xmin: float = 0.0, xmax: float = 1.0, device="cuda"):
        self.n = int(n)
        self.xmin, self.xmax = float(xmin), float(xmax)
        self.xold1, self.xold2, self.low, self.upp = (
            torch.zeros(self.n, dtype=torch.float64, device=device) for _ in range(4))
        self.device = self.xold1.device  # with its index ("cuda" -> "cuda:0"), as tensors report it
        self.iteration = 0

    def step(self, x: torch.Tensor, df: torch.Tensor) -> None:
        """Moves x (contiguous float64 device tensor of n values) in place, ascending along df."""
        if x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != self.n or x.device != self.device:
            raise ValueError("x must be a contiguous float64 tensor of n values on the solver's device")
        df = df.detach().to(self.device, torch.float64).contiguous()
        if df.numel() != self.n:
            raise ValueError("gradient size does not match the design")
        B.pc_mma_step(self.n, x.data_ptr(), df.data_ptr(), self.xold1.data_ptr(), self.xold2.data_ptr(),
                      self.low.data_ptr(), self.upp.data_ptr(), self.iteration, self.xmin, self.xmax,
                      torch.cuda.current_stream(self.device).cuda_stream)
        self.iteration += 1


def maximize_gap(solver: BandSolver, rho: torch.Tensor, n_lower: int, beta: float, steps: int):
    """Optimization loop of eq. topopt on the smooth (KS) gap between bands n_lower and n_lower+1:
    band structure, gap and adjoint gradient, then one MMA design update, `steps` times.  Returns
    the final design (n0, n1, n2) and the gap before each step and after the last."""
    x = rho.detach().to(solver.device, torch.float64).contiguous().clone().view(-1)
    opt = MMA(x.numel(), device=solver.device)
    history = []
    for _ in range(steps):
        solver.set_design(x)
        solver.bands()
        g, grad = solver.gap_ks_and_grad(n_lower, beta)
        history.append(float(g.item()))
        opt.step(x, grad.view(-1))
    solver.set_design(x)
    solver.bands()
    g, _ = solver.gap_ks_and_grad(n_lower, beta, need_grad=False)
    history.append(float(g.item()))
    return x.view(solver.n), history
