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
                 tol=0.0, max_iter=0, device="cuda", law="compliance"):
        if isinstance(precision, str):
            precision = {"fp64": B.PC_FP64, "mixed": B.PC_MIXED}[precision]
        self.device = torch.device(device)
        self.n = tuple(int(x) for x in n)
        self.nbands = int(nbands)
        self.params = B.make_params(lattice, n, M, nbands, phase1, phase0, penal, precision, a, tol, max_iter, law)
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

    def set_warm_start(self, on: bool = True) -> None:
        """Start each bands() from the previous call's final Ritz block (same k-points)."""
        B.pc_set_warm_start(self.ctx, on)

    def import_block(self, block: np.ndarray) -> None:
        """Start the next bands() from a block exported by export(PC_EXPORT_BLOCK)."""
        B.pc_import_block(self.ctx, block)

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


class DesignMap:
    """Reduced design field -> element densities (pc_design_*): linear-weight average of the
    design nodes within the radius, Heaviside projection at sharpness beta, optional SC octant
    symmetry.  The radius defaults to 1.4 element edges (|a_1| / n_1)."""

    def __init__(self, lattice, n, spacing: int = 2, radius: float | None = None, octant: bool = False,
                 a: float = 1.0, device="cuda"):
        import math
        self.device = torch.device(device)
        self.n = tuple(int(v) for v in n)
        if radius is None:
            edge = {"sc": 1.0, "bcc": math.sqrt(3.0) / 2.0, "fcc": math.sqrt(2.0) / 2.0}[lattice] * a / self.n[0]
            radius = 1.4 * edge
        cell = B.make_params(lattice, self.n, 1, 1, {"rho": 1.0, "E": 1.0, "nu": 0.3},
                             {"rho": 1.0, "E": 1.0, "nu": 0.3}, a=a)
        self.handle = B.pc_design_create(cell, B.make_design_params(spacing, radius, octant))
        self.nvars = B.pc_design_nvars(self.handle)

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def project(self, x: torch.Tensor, beta: float, out: torch.Tensor | None = None) -> torch.Tensor:
        x = x.detach().to(self.device, torch.float64).contiguous()
        if x.numel() != self.nvars:
            raise ValueError("x must hold nvars values")
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device=self.device)
        self._x = x
        B.pc_design_project(self.handle, x.data_ptr(), beta, out.data_ptr(), self._stream())
        return out

    def backprop(self, g_rho: torch.Tensor) -> torch.Tensor:
        """d/dx from d/drho, at the x and beta of the last project()."""
        g_rho = g_rho.detach().to(self.device, torch.float64).contiguous()
        gx = torch.empty(self.nvars, dtype=torch.float64, device=self.device)
        B.pc_design_backprop(self.handle, g_rho.data_ptr(), gx.data_ptr(), self._stream())
        return gx

    def close(self):
        if getattr(self, "handle", 0):
            B.pc_design_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ProjectFn(torch.autograd.Function):
    """x (nvars) -> rho (n0, n1, n2) through a DesignMap at sharpness beta; backward by the
    map's chain rule (the forward is re-run first, so interleaved calls stay consistent)."""

    @staticmethod
    def forward(ctx, x, dmap: DesignMap, beta: float):
        ctx.save_for_backward(x.detach().clone())
        ctx.dmap, ctx.beta = dmap, beta
        return dmap.project(x, beta)

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        ctx.dmap.project(x, ctx.beta)
        return ctx.dmap.backprop(g), None, None


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


def heaviside_schedule(step: int, every: int, start: float = 1.0, factor: float = 2.0, cap: float = 64.0) -> float:
    """Continuation of the projection sharpness: start (the paper's beta = 1), multiplied by
    factor every `every` steps, at most cap."""
    return min(cap, start * factor ** (step // max(1, every)))


def maximize_gap(solver: BandSolver, rho: torch.Tensor, n_lower: int, beta: float, steps: int,
                 design: DesignMap | None = None, beta_every: int = 0):
    """Optimization loop of eq. topopt on the smooth (KS) gap between bands n_lower and n_lower+1:
    band structure, gap and adjoint gradient, then one MMA design update, `steps` times.  Without
    a design map the variables are the densities (rho, shape n); with one they are its free
    variables (rho, nvars values in [0, 1]), the densities are their projection at the sharpness
    heaviside_schedule(step, beta_every) (beta_every = 0: 1 throughout) and the gradient is carried
    back through the map.  Returns the final variables and the gap before each step and after
    the last.  The gradient's relative error is about the final residual of the bands n_lower and
    n_lower+1: in the mixed form, build the solver with tol = 1e-4 for a 1e-4 gradient."""
    x = rho.detach().to(solver.device, torch.float64).contiguous().clone().view(-1)
    opt = MMA(x.numel(), device=solver.device)
    history = []

    def evaluate(step, need_grad):
        if design is None:
            solver.set_design(x)
        else:
            hb = heaviside_schedule(step, beta_every) if beta_every > 0 else 1.0
            solver.set_design(design.project(x, hb))
        solver.bands()
        g, grad = solver.gap_ks_and_grad(n_lower, beta, need_grad=need_grad)
        if need_grad and design is not None:
            grad = design.backprop(grad)
        return g, grad

    for step in range(steps):
        g, grad = evaluate(step, True)
        history.append(float(g.item()))
        opt.step(x, grad.view(-1))
    g, _ = evaluate(steps, False)
    history.append(float(g.item()))
    return (x.view(solver.n) if design is None else x), history


class BatchSolver:
    """Designs of different lattices, grids, cutoffs and k-points evaluated in one call each
    (pc_batch_*).  `designs`: objects with lattice, n, M, nbands, phase1, phase0, Q, penal and a
    (e.g. workloads.Workload).  workers / kgroups: concurrency of the batch (see autotune); the
    packed outputs are returned as per-design views."""

    def __init__(self, designs, precision=B.PC_MIXED, workers: int = 4, kgroups: int = 0, device="cuda",
                 law="compliance"):
        if isinstance(precision, str):
            precision = {"fp64": B.PC_FP64, "mixed": B.PC_MIXED}[precision]
        self.device = torch.device(device)
        self.designs = list(designs)
        self.params = [B.make_params(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.penal, precision,
                                     getattr(w, "a", 1.0), law=law) for w in self.designs]
        Q = np.concatenate([np.asarray(w.Q, dtype=np.float64) for w in self.designs], axis=0)
        self.nk = [int(np.asarray(w.Q).shape[0]) for w in self.designs]
        self.ne = [int(np.prod(w.n)) for w in self.designs]
        self.nb = [int(w.nbands) for w in self.designs]
        self.handle = B.pc_batch_create(self.params, Q, self.nk, workers, kgroups)
        self.off_rho = np.concatenate([[0], np.cumsum(self.ne)]).astype(int)
        self.off_om = np.concatenate([[0], np.cumsum([k * b for k, b in zip(self.nk, self.nb)])]).astype(int)

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def set_designs(self, rhos) -> None:
        """rhos: one density tensor per design (any shape with n0 n1 n2 values) or a packed tensor."""
        if isinstance(rhos, torch.Tensor):
            packed = rhos.detach().to(self.device, torch.float64).contiguous().view(-1)
        else:
            packed = torch.cat([torch.as_tensor(r).to(self.device, torch.float64).reshape(-1) for r in rhos])
        if packed.numel() != self.off_rho[-1]:
            raise ValueError("densities do not match the designs' grids")
        self._rho = packed
        B.pc_batch_set_designs(self.handle, packed.data_ptr(), self._stream())

    def bands(self):
        om = torch.empty(int(self.off_om[-1]), dtype=torch.float64, device=self.device)
        B.pc_batch_bands(self.handle, om.data_ptr(), self._stream())
        self._om = om
        return [om[self.off_om[d]:self.off_om[d + 1]].view(self.nk[d], self.nb[d]) for d in range(len(self.designs))]

    def gap_and_grad(self, n_lower=None, mode: int = B.PC_GAP_OMEGA, weights=None, need_grad: bool = True):
        nd = len(self.designs)
        gap = torch.empty(nd, dtype=torch.float64, device=self.device)
        grad = torch.empty(int(self.off_rho[-1]), dtype=torch.float64, device=self.device) if need_grad else None
        wptr = 0
        if weights is not None:
            wt = torch.cat([torch.as_tensor(w).to(self.device, torch.float64).reshape(-1) for w in weights])
            self._w = wt
            wptr = wt.data_ptr()
        nl = np.ones(nd, dtype=np.int32) if n_lower is None else np.asarray(n_lower, dtype=np.int32)
        B.pc_batch_gap_and_grad(self.handle, nl, mode, wptr, gap.data_ptr(), grad.data_ptr() if need_grad else 0,
                                self._stream())
        grads = None
        if need_grad:
            grads = [grad[self.off_rho[d]:self.off_rho[d + 1]].view(self.designs[d].n) for d in range(nd)]
        return gap, grads

    def stats(self, design: int):
        return B.pc_batch_get_stats(self.handle, design)

    def close(self):
        if getattr(self, "handle", 0):
            B.pc_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
