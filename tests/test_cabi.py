"""C-ABI checks that need no GPU: the library loads, exports every declared entry point,
and rejects bad arguments on the host before touching the device."""
import os
import re

import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1603_06855_gb300 import binding as B, build_lib
    if not os.path.exists(B.LIB_PATH):
        build_lib.build()
    return B


def test_header_symbols_exported():
    B = _lib()
    header = open(os.path.join(ROOT, "include", "phononic.h")).read()
    declared = set(re.findall(r"\b(pc_[a-z_]+)\s*\(", header))
    assert declared == set(B.EXPORTED)
    lib = B.load()
    for name in declared:
        assert hasattr(lib, name)


def test_strerror():
    B = _lib()
    assert B.pc_strerror(0) == "PC_OK"
    assert B.pc_strerror(2) == "PC_EALIAS"
    assert B.pc_strerror(99) == "PC_UNKNOWN"


def _params(**kw):
    B = _lib()
    base = dict(lattice="sc", n=(8, 8, 8), M=1, nbands=6, phase1=wl.TUNGSTEN_CARBIDE, phase0=wl.EPOXY)
    base.update(kw)
    return B.make_params(**base)


@pytest.mark.parametrize("kw,code", [
    (dict(M=0), 1), (dict(M=6), 1), (dict(nbands=0), 1), (dict(nbands=25), 1), (dict(lattice=7), 1),
    (dict(n=(8, 0, 8)), 1), (dict(penal=0.5), 1), (dict(precision=3), 1), (dict(a=-1.0), 1),
    (dict(phase1=dict(rho=1.0, E=1.0, nu=0.5)), 1), (dict(phase0=dict(rho=-1.0, E=1.0, nu=0.3)), 1),
    (dict(n=(8, 4, 8), M=2), 2), (dict(n=(2, 8, 8), M=1), 2), (dict(law=2), 1), (dict(law=-1), 1),
])
def test_create_rejects_bad_parameters(kw, code):
    B = _lib()
    assert B.pc_create_rc(_params(**kw)) == code


def test_null_handles_rejected():
    B = _lib()
    lib = B.load()
    assert lib.pc_set_kpoints(None, None, 3) == B.PC_EINVAL
    assert lib.pc_bands(None, None, None) == B.PC_EINVAL
    assert lib.pc_gap_and_grad(None, 1, 0, None, None, None, None) == B.PC_EINVAL
    assert lib.pc_clear_status(None) == B.PC_EINVAL
    assert lib.pc_set_warm_start(None, 1) == B.PC_EINVAL
    assert lib.pc_import_block(None, None, 0) == B.PC_EINVAL
    lib.pc_destroy(None)


def test_kpoint_count_limit():
    """nk outside [1, PC_MAX_KPOINTS] (the wavevector index is a launch grid dimension) is
    rejected before the context is used: the placeholder handle is never dereferenced."""
    import ctypes
    B = _lib()
    lib = B.load()
    hdr = open(os.path.join(ROOT, "include", "phononic.h")).read()
    limit = int(re.search(r"#define PC_MAX_KPOINTS\s+(\d+)", hdr).group(1))
    assert limit == 65535
    q = ctypes.create_string_buffer(24 * (limit + 1))
    placeholder = ctypes.create_string_buffer(64)
    for nk in (0, -1, limit + 1):
        assert lib.pc_set_kpoints(ctypes.addressof(placeholder), ctypes.addressof(q), nk) == B.PC_EINVAL


def test_mma_step_rejects_bad_arguments():
    """pc_mma_step validates its arguments on the host before launching anything; the
    placeholder buffers below are never dereferenced."""
    import ctypes
    B = _lib()
    lib = B.load()
    buf = ctypes.create_string_buffer(64)
    p = ctypes.addressof(buf)
    good = dict(n=4, x=p, df=p, x1=p, x2=p, lo=p, up=p, it=0, xmin=0.0, xmax=1.0)

    def call(**kw):
        a = dict(good, **kw)
        return lib.pc_mma_step(a["n"], a["x"], a["df"], a["x1"], a["x2"], a["lo"], a["up"], a["it"],
                               a["xmin"], a["xmax"], None)

    for bad in (dict(n=0), dict(n=-3), dict(x=None), dict(df=None), dict(x1=None), dict(x2=None),
                dict(lo=None), dict(up=None), dict(it=-1), dict(xmax=0.0), dict(xmin=2.0),
                dict(xmin=float("nan")), dict(xmax=float("inf"))):
        assert call(**bad) == B.PC_EINVAL, bad


@pytest.mark.parametrize("kw,code", [
    (dict(phase1=dict(rho=1.0, E=1.0, nu=0.5)), 1), (dict(phase0=dict(rho=1.0, E=float("nan"), nu=0.3)), 1),
    (dict(phase0=dict(rho=float("inf"), E=1.0, nu=0.3)), 1), (dict(phase1=dict(rho=1.0, E=1.0, nu=-1.0)), 1),
    (dict(penal=float("inf")), 1), (dict(penal=0.5), 1), (dict(M=0), 1), (dict(M=6), 1),
    (dict(n=(300, 8, 8)), 1), (dict(n=(8, 0, 8)), 1), (dict(law=3), 1),
    (dict(n=(8, 4, 8), M=2), 2),
    (dict(n=(48, 48, 48), M=2), 9), (dict(n=(64, 64, 64)), 9),
])
def test_noalloc_rejects_bad_parameters_on_host(kw, code):
    """pc_structure_factors_noalloc applies pc_create's parameter rules and its own size limit
    before any CUDA call (the placeholder pointers below are never dereferenced)."""
    import ctypes
    B = _lib()
    lib = B.load()
    buf = ctypes.create_string_buffer(64)
    p = _params(**kw)
    assert lib.pc_structure_factors_noalloc(ctypes.byref(p), ctypes.addressof(buf), ctypes.addressof(buf),
                                            None) == code
    assert lib.pc_structure_factors_noalloc(ctypes.byref(p), None, ctypes.addressof(buf), None) == B.PC_EINVAL


@pytest.mark.parametrize("lattice,n,spacing,rad,octant", [
    ("sc", (8, 8, 8), 3, 2.0, 0), ("sc", (9, 8, 8), 2, 2.0, 0), ("bcc", (8, 8, 8), 2, 2.0, 1),
    ("sc", (10, 10, 10), 2, 2.0, 1),   # the octant needs an even design grid (5 nodes per axis)
    ("sc", (8, 8, 8), 2, 0.3, 0),      # no node within the radius
    ("sc", (8, 8, 8), 2, 7.0, 0),      # the radius reaches a node's periodic image
    ("sc", (8, 8, 8), 2, -1.0, 0), ("sc", (8, 8, 8), 2, 2.0, 2),
])
def test_design_create_rejects_bad_parameters(lattice, n, spacing, rad, octant):
    """pc_design_create validates on the host before allocating anything."""
    B = _lib()
    cell = _params(lattice=lattice, n=n)
    dp = B.make_design_params(spacing, rad / n[0], bool(octant))
    dp.octant = octant
    rc, h = B.pc_design_create_rc(cell, dp)
    assert rc == B.PC_EINVAL and h == 0


def test_batch_create_rejects_bad_arguments():
    """pc_batch_create checks its counts before creating any context, and a design with bad
    parameters fails in pc_create's own host checks (no device memory is touched)."""
    import numpy as np
    B = _lib()
    good = _params()
    q = np.zeros((4, 3))
    for workers, kgroups, nk in ((0, 0, [2, 2]), (17, 0, [2, 2]), (2, 7, [2, 2]), (2, -1, [2, 2]), (2, 0, [0, 4])):
        rc, h = B.pc_batch_create_rc([good, good], q, nk, workers, kgroups)
        assert rc == B.PC_EINVAL and h == 0
    rc, h = B.pc_batch_create_rc([_params(M=0)], q[:2], [2], 1, 0)
    assert rc == B.PC_EINVAL and h == 0
    lib = B.load()
    assert lib.pc_batch_bands(None, None, None) == B.PC_EINVAL
    assert lib.pc_batch_set_designs(None, None, None) == B.PC_EINVAL
    lib.pc_batch_destroy(None)
