"""ctypes binding of libphononic.so: the C entry points under their own names, plus a thin
torch-facing wrapper.  Argument marshalling only: every step of the band and adjoint
path runs in the library's CUDA kernels.  Importing this module raises if the library
has not been built; there is no fallback."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphononic.so")

PC_OK, PC_EINVAL, PC_EALIAS, PC_ENOMEM, PC_ECUDA, PC_ESTATE, PC_ENOCONV, PC_EDOMAIN, PC_ETIMEOUT, PC_ETOOBIG = range(10)
PC_SC, PC_BCC, PC_FCC = 0, 1, 2
PC_FP64, PC_MIXED = 0, 1
PC_GAP_OMEGA, PC_GAP_LAMBDA, PC_GRAD_ALLBANDS = 0, 1, 2
PC_CLUSTER_TOL_FP64, PC_CLUSTER_TOL_MIXED = 1e-8, 1e-6
PC_EXPORT_SFAC, PC_EXPORT_TOEP, PC_EXPORT_WINV, PC_EXPORT_EIGVEC, PC_EXPORT_LAMBDA, PC_EXPORT_WEIGHT, PC_EXPORT_BLOCK = range(7)
PC_LAW_COMPLIANCE, PC_LAW_YOUNG = 0, 1
LAWS = {"compliance": PC_LAW_COMPLIANCE, "young": PC_LAW_YOUNG}
LATTICES = {"sc": PC_SC, "bcc": PC_BCC, "fcc": PC_FCC}


class pc_material(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("E", ctypes.c_double), ("nu", ctypes.c_double)]


class pc_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("a", ctypes.c_double),
        ("n", ctypes.c_int * 3),
        ("M", ctypes.c_int),
        ("phase1", pc_material),
        ("phase0", pc_material),
        ("penal", ctypes.c_double),
        ("nbands", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("law", ctypes.c_int),
    ]


class pc_design_params(ctypes.Structure):
    _fields_ = [("spacing", ctypes.c_int), ("radius", ctypes.c_double), ("octant", ctypes.c_int)]


class pc_stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("unconverged_k", ctypes.c_int),
        ("nk", ctypes.c_int),
        ("N", ctypes.c_int),
        ("block", ctypes.c_int),
        ("max_residual", ctypes.c_double),
        ("ms_setup", ctypes.c_double),
        ("ms_bands", ctypes.c_double),
        ("ms_grad", ctypes.c_double),
        ("launches", ctypes.c_longlong),
        ("ms_rr_gemm", ctypes.c_double),
        ("rr_gemm_launches", ctypes.c_longlong),
        ("rr_gemm_flops", ctypes.c_double),
        ("ms_iter_apply", ctypes.c_double),
        ("iter_apply_calls", ctypes.c_longlong),
        ("iter_apply_flops", ctypes.c_double),
        ("ms_small", ctypes.c_double),
        ("ms_grad_kernels", ctypes.c_double),
        ("ms_gram", ctypes.c_double),
        ("gram_launches", ctypes.c_longlong),
        ("gram_flops", ctypes.c_double),
        ("gram_bytes", ctypes.c_double),
        ("ms_update", ctypes.c_double),
        ("update_launches", ctypes.c_longlong),
        ("update_flops", ctypes.c_double),
        ("update_bytes", ctypes.c_double),
        ("ms_iteration_loop", ctypes.c_double),
        ("ms_final_rr", ctypes.c_double),
        ("small_flops", ctypes.c_double),
        ("grad_pairs", ctypes.c_longlong),
        ("grad_flops_per_pair", ctypes.c_double),
        ("ms_host_idle", ctypes.c_double),
        ("rr_sliced", ctypes.c_int),
        ("small_calls", ctypes.c_longlong),
    ]


EXPORTED = ["pc_create", "pc_set_kpoints", "pc_set_design", "pc_bands", "pc_gap_and_grad", "pc_gap_ks_and_grad",
            "pc_get_stats",
            "pc_clear_status", "pc_set_profiling", "pc_probe", "pc_destroy", "pc_strerror", "pc_export",
            "pc_apply_operator", "pc_check_tensor_kernels", "pc_structure_factors_noalloc", "pc_mma_step",
            "pc_design_create", "pc_design_nvars", "pc_design_project", "pc_design_backprop", "pc_design_destroy",
            "pc_set_warm_start", "pc_import_block", "pc_batch_create", "pc_batch_set_designs", "pc_batch_bands",
            "pc_batch_gap_and_grad", "pc_batch_get_stats", "pc_batch_destroy"]

_lib = None


def load(path: str = LIB_PATH):
    """Loads the compiled library (raises OSError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: run paper_1603_06855_gb300.build_lib.build() first")
    lib = ctypes.CDLL(path)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    lib.pc_create.argtypes = [ctypes.POINTER(pc_params), ctypes.POINTER(P)]
    lib.pc_set_kpoints.argtypes = [P, P, I]
    lib.pc_set_design.argtypes = [P, P, P]
    lib.pc_bands.argtypes = [P, P, P]
    lib.pc_gap_and_grad.argtypes = [P, I, I, P, P, P, P]
    lib.pc_gap_ks_and_grad.argtypes = [P, I, D, P, P, P]
    lib.pc_get_stats.argtypes = [P, ctypes.POINTER(pc_stats)]
    lib.pc_clear_status.argtypes = [P]
    lib.pc_set_profiling.argtypes = [P, I]
    lib.pc_probe.argtypes = [I, ctypes.POINTER(D)]
    lib.pc_destroy.argtypes = [P]
    lib.pc_destroy.restype = None
    lib.pc_strerror.argtypes = [I]
    lib.pc_strerror.restype = ctypes.c_char_p
    lib.pc_export.argtypes = [P, I, P, LL, ctypes.POINTER(LL)]
    lib.pc_apply_operator.argtypes = [P, I, I, P, P, P, P]
    lib.pc_structure_factors_noalloc.argtypes = [ctypes.POINTER(pc_params), P, P, P]
    lib.pc_check_tensor_kernels.argtypes = [I, I, I, I, I, ctypes.POINTER(ctypes.c_double)]
    lib.pc_mma_step.argtypes = [LL, P, P, P, P, P, P, I, D, D, P]
    lib.pc_design_create.argtypes = [ctypes.POINTER(pc_params), ctypes.POINTER(pc_design_params), ctypes.POINTER(P)]
    lib.pc_design_nvars.argtypes = [P]
    lib.pc_design_project.argtypes = [P, P, D, P, P]
    lib.pc_design_backprop.argtypes = [P, P, P, P]
    lib.pc_design_destroy.argtypes = [P]
    lib.pc_set_warm_start.argtypes = [P, I]
    lib.pc_batch_create.argtypes = [P, I, P, P, I, I, ctypes.POINTER(P)]
    lib.pc_batch_set_designs.argtypes = [P, P, P]
    lib.pc_batch_bands.argtypes = [P, P, P]
    lib.pc_batch_gap_and_grad.argtypes = [P, P, I, P, P, P, P]
    lib.pc_batch_get_stats.argtypes = [P, I, ctypes.POINTER(pc_stats)]
    lib.pc_batch_destroy.argtypes = [P]
    lib.pc_import_block.argtypes = [P, P, LL]
    for name in EXPORTED:
        if name not in ("pc_destroy", "pc_strerror", "pc_design_destroy", "pc_design_nvars", "pc_batch_destroy"):
            getattr(lib, name).restype = I
    lib.pc_design_nvars.restype = LL
    lib.pc_design_destroy.restype = None
    lib.pc_batch_destroy.restype = None
    _lib = lib
    return lib


def pc_strerror(code: int) -> str:
    return load().pc_strerror(code).decode()


class PhononicError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {pc_strerror(code)} ({code})")
        self.code = code


def _check(rc: int, where: str):
    if rc != PC_OK:
        raise PhononicError(rc, where)


def make_params(lattice, n, M, nbands, phase1, phase0, penal=1.0, precision=PC_FP64, a=1.0, tol=0.0,
                max_iter=0, law=PC_LAW_COMPLIANCE) -> pc_params:
    p = pc_params()
    p.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    p.a = float(a)
    for i in range(3):
        p.n[i] = int(n[i])
    p.M = int(M)
    p.phase1 = pc_material(phase1["rho"], phase1["E"], phase1["nu"])
    p.phase0 = pc_material(phase0["rho"], phase0["E"], phase0["nu"])
    p.penal = float(penal)
    p.nbands = int(nbands)
    p.precision = int(precision)
    p.tol = float(tol)
    p.max_iter = int(max_iter)
    p.law = LAWS[law] if isinstance(law, str) else int(law)
    return p


def pc_create(params: pc_params) -> int:
    h = ctypes.c_void_p()
    _check(load().pc_create(ctypes.byref(params), ctypes.byref(h)), "pc_create")
    return h.value


def pc_create_rc(params: pc_params) -> int:
    """Return code only (for argument-validation tests; frees any context created)."""
    h = ctypes.c_void_p()
    rc = load().pc_create(ctypes.byref(params), ctypes.byref(h))
    if rc == PC_OK and h.value:
        load().pc_destroy(h)
    return rc


def pc_set_kpoints(ctx: int, q_host) -> None:
    import numpy as np
    q = np.ascontiguousarray(q_host, dtype=np.float64)
    _check(load().pc_set_kpoints(ctx, q.ctypes.data, q.shape[0]), "pc_set_kpoints")


def pc_set_design(ctx: int, rho_ptr: int, stream: int = 0) -> None:
    _check(load().pc_set_design(ctx, rho_ptr, stream), "pc_set_design")


def pc_bands(ctx: int, omega_ptr: int, stream: int = 0) -> None:
    _check(load().pc_bands(ctx, omega_ptr, stream), "pc_bands")


def pc_gap_and_grad(ctx: int, n_lower: int, mode: int, w_ptr: int, gap_ptr: int, grad_ptr: int,
                    stream: int = 0) -> None:
    _check(load().pc_gap_and_grad(ctx, n_lower, mode, w_ptr, gap_ptr, grad_ptr, stream), "pc_gap_and_grad")


def pc_gap_ks_and_grad(ctx: int, n_lower: int, beta: float, gap_ptr: int, grad_ptr: int, stream: int = 0) -> None:
    _check(load().pc_gap_ks_and_grad(ctx, n_lower, beta, gap_ptr, grad_ptr, stream), "pc_gap_ks_and_grad")


def pc_mma_step(n: int, x_ptr: int, df_ptr: int, xold1_ptr: int, xold2_ptr: int, low_ptr: int, upp_ptr: int,
                iteration: int, xmin: float = 0.0, xmax: float = 1.0, stream: int = 0) -> None:
    _check(load().pc_mma_step(n, x_ptr, df_ptr, xold1_ptr, xold2_ptr, low_ptr, upp_ptr, iteration, xmin, xmax,
                              stream), "pc_mma_step")


def pc_get_stats(ctx: int) -> pc_stats:
    st = pc_stats()
    load().pc_get_stats(ctx, ctypes.byref(st))
    return st


def pc_clear_status(ctx: int) -> None:
    _check(load().pc_clear_status(ctx), "pc_clear_status")


def pc_set_profiling(ctx: int, on: bool) -> None:
    _check(load().pc_set_profiling(ctx, 1 if on else 0), "pc_set_profiling")


def pc_probe(what: int) -> float:
    v = ctypes.c_double()
    _check(load().pc_probe(what, ctypes.byref(v)), "pc_probe")
    return v.value


def pc_destroy(ctx: int) -> None:
    load().pc_destroy(ctx)


def pc_export(ctx: int, which: int):
    import numpy as np
    n = ctypes.c_longlong()
    _check(load().pc_export(ctx, which, None, 0, ctypes.byref(n)), "pc_export")
    out = np.empty(n.value, dtype=np.float64)
    _check(load().pc_export(ctx, which, out.ctypes.data, n.value, ctypes.byref(n)), "pc_export")
    return out


def pc_apply_operator(ctx: int, k: int, ncols: int, x_ptr: int, ax_ptr: int, ox_ptr: int, stream: int = 0):
    _check(load().pc_apply_operator(ctx, k, ncols, x_ptr, ax_ptr, ox_ptr, stream), "pc_apply_operator")


def pc_check_tensor_kernels(what: int, nk: int, m: int, nblk: int, n3: int) -> float:
    """Tensor-core vs CUDA-core Gram (what=0) or basis update (what=1), or the sliced FP64-accurate
    product vs the FP64 GEMM (what=3, n3 = N, nk * m columns): max relative difference."""
    err = ctypes.c_double(-1.0)
    _check(load().pc_check_tensor_kernels(what, nk, m, nblk, n3, ctypes.byref(err)), "pc_check_tensor_kernels")
    return err.value


def pc_structure_factors_noalloc(params: pc_params, rho_ptr: int, sfac_ptr: int, stream: int = 0) -> int:
    """Allocation-free structure factors (return code; 0 on success)."""
    return load().pc_structure_factors_noalloc(ctypes.byref(params), rho_ptr, sfac_ptr, stream)


def make_design_params(spacing: int = 2, radius: float = 0.0, octant: bool = False) -> pc_design_params:
    dp = pc_design_params()
    dp.spacing = int(spacing)
    dp.radius = float(radius)
    dp.octant = 1 if octant else 0
    return dp


def pc_design_create_rc(cell: pc_params, dp: pc_design_params):
    """(return code, handle or 0)."""
    h = ctypes.c_void_p()
    rc = load().pc_design_create(ctypes.byref(cell), ctypes.byref(dp), ctypes.byref(h))
    return rc, (h.value or 0)


def pc_design_create(cell: pc_params, dp: pc_design_params) -> int:
    rc, h = pc_design_create_rc(cell, dp)
    _check(rc, "pc_design_create")
    return h


def pc_design_nvars(d: int) -> int:
    return int(load().pc_design_nvars(d))


def pc_design_project(d: int, x_ptr: int, beta: float, rho_ptr: int, stream: int = 0) -> None:
    _check(load().pc_design_project(d, x_ptr, float(beta), rho_ptr, stream), "pc_design_project")


def pc_design_backprop(d: int, g_rho_ptr: int, g_x_ptr: int, stream: int = 0) -> None:
    _check(load().pc_design_backprop(d, g_rho_ptr, g_x_ptr, stream), "pc_design_backprop")


def pc_design_destroy(d: int) -> None:
    if d:
        load().pc_design_destroy(d)


def pc_set_warm_start(ctx: int, on: bool) -> None:
    _check(load().pc_set_warm_start(ctx, 1 if on else 0), "pc_set_warm_start")


def pc_import_block(ctx: int, block) -> None:
    import numpy as np
    b = np.ascontiguousarray(block, dtype=np.float64)
    _check(load().pc_import_block(ctx, b.ctypes.data, b.size // 2), "pc_import_block")


def pc_batch_create_rc(params, q_host, nk, workers: int = 1, kgroups: int = 0):
    """(return code, handle or 0) for a list of pc_params, concatenated k-points and counts."""
    import numpy as np
    arr = (pc_params * len(params))(*params)
    q = np.ascontiguousarray(q_host, dtype=np.float64)
    counts = np.ascontiguousarray(nk, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = load().pc_batch_create(ctypes.addressof(arr), len(params), q.ctypes.data, counts.ctypes.data, int(workers),
                                int(kgroups), ctypes.byref(h))
    return rc, (h.value or 0)


def pc_batch_create(params, q_host, nk, workers: int = 1, kgroups: int = 0) -> int:
    rc, h = pc_batch_create_rc(params, q_host, nk, workers, kgroups)
    _check(rc, "pc_batch_create")
    return h


def pc_batch_set_designs(b: int, rho_ptr: int, stream: int = 0) -> None:
    _check(load().pc_batch_set_designs(b, rho_ptr, stream), "pc_batch_set_designs")


def pc_batch_bands(b: int, omega_ptr: int, stream: int = 0) -> None:
    _check(load().pc_batch_bands(b, omega_ptr, stream), "pc_batch_bands")


def pc_batch_gap_and_grad(b: int, n_lower, mode: int, w_ptr: int, gap_ptr: int, grad_ptr: int, stream: int = 0):
    import numpy as np
    nl = np.ascontiguousarray(n_lower, dtype=np.int32)
    _check(load().pc_batch_gap_and_grad(b, nl.ctypes.data, mode, w_ptr, gap_ptr, grad_ptr, stream),
           "pc_batch_gap_and_grad")


def pc_batch_get_stats(b: int, design: int) -> pc_stats:
    st = pc_stats()
    load().pc_batch_get_stats(b, design, ctypes.byref(st))
    return st


def pc_batch_destroy(b: int) -> None:
    if b:
        load().pc_batch_destroy(b)
