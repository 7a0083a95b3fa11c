"""The ctypes mirrors of the C ABI (binding.py) match include/phononic.h: a small C program
compiled against the header prints sizeof and every field's offsetof of the structs and the value
of every constant, which must equal the ctypes layout and the binding's constants; every entry
point's ctypes argument and return types agree with its prototype.  CPU only (gcc); a mismatch
would make the binding read or write the wrong bytes without any error."""
import ctypes
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1603_06855_gb300 import binding as B  # noqa: E402

STRUCTS = [B.pc_material, B.pc_params, B.pc_design_params, B.pc_stats]


def _c_layout(tmp_path):
    lines = ['#include "phononic.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, value = line.split()
        layout[(name, key)] = int(value)
    return layout


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for st in STRUCTS:
        name = st.__name__
        assert layout[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert layout[(name, field)] == getattr(st, field).offset, (name, field)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_constants_match_the_header(tmp_path):
    """Every value macro of include/phononic.h (error codes, lattices, forms, laws, gap modes,
    export selectors, cluster windows) has a binding constant of the same name and value, as the
    C compiler evaluates it.  PC_MAX_KPOINTS is a limit the library checks itself (test_cabi)."""
    import re
    hdr = open(os.path.join(ROOT, "include", "phononic.h")).read()
    names = [n for n in re.findall(r"^#define\s+(PC_\w+)\s+\S", hdr, re.M) if n != "PC_MAX_KPOINTS"]
    assert len(names) >= 25
    lines = ['#include "phononic.h"', "#include <stdio.h>", "int main(void) {"]
    lines += [f'  printf("{n} %.17g\\n", (double)({n}));' for n in names]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        name, value = line.split()
        assert hasattr(B, name), name
        assert float(getattr(B, name)) == float(value), (name, getattr(B, name), value)


def _c_kind(ctype: str):
    """Kind of a C parameter or return type: 'int', 'double', 'long long', 'void', or
    ('ptr', pointee) with pointee the base type name ('**' pointers give ('ptr', 'void*'))."""
    t = " ".join(ctype.replace("const", " ").split())
    if t.count("*") >= 2:
        return ("ptr", "void*")
    if "*" in t:
        return ("ptr", t.replace("*", "").strip())
    return t


def _ctypes_kind(ct):
    import ctypes
    if ct is None:
        return "void"
    simple = {ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_longlong: "long long"}
    if ct in simple:
        return simple[ct]
    if ct in (ctypes.c_void_p, ctypes.c_char_p):
        return ("ptr", None)
    if hasattr(ct, "_type_") and isinstance(ct._type_, type):  # POINTER(x)
        inner = ct._type_
        if inner is ctypes.c_void_p:
            return ("ptr", "void*")
        names = {ctypes.c_double: "double", ctypes.c_longlong: "long long", ctypes.c_int: "int"}
        return ("ptr", names.get(inner, inner.__name__))
    raise AssertionError(f"unexpected ctypes type {ct!r}")


def test_binding_signatures_match_the_header():
    """Every entry point of include/phononic.h has ctypes argtypes and restype in binding.load()
    that agree with its prototype: same arity, int / double / long long by width, pointers either
    untyped (an address, e.g. of a ctypes array of structs) or typed with the same base type or
    struct, out-handles as POINTER(c_void_p).  A mismatch would pass wrong values to the library
    without any error."""
    import re
    if not os.path.exists(B.LIB_PATH):
        from paper_1603_06855_gb300 import build_lib
        build_lib.build()
    lib = B.load()
    hdr = re.sub(r"/\*.*?\*/", " ", open(os.path.join(ROOT, "include", "phononic.h")).read(), flags=re.S)
    protos = re.findall(r"^(int|void|long long|const char\s*\*)\s*(pc_\w+)\(([^)]*)\);", hdr, re.M)
    assert len(protos) >= 30
    for ret, name, params in protos:
        fn = getattr(lib, name)
        params = " ".join(params.split())
        cparams = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        ctypes_args = fn.argtypes
        assert ctypes_args is not None, name
        assert len(ctypes_args) == len(cparams), (name, len(ctypes_args), cparams)
        for cp, ct in zip(cparams, ctypes_args):
            ckind = _c_kind(cp.rsplit(" ", 1)[0] if not cp.endswith("*") else cp)
            pkind = _ctypes_kind(ct)
            if isinstance(ckind, tuple):
                assert isinstance(pkind, tuple), (name, cp, ct)
                if ckind[1] == "void*":  # an out-handle: POINTER(c_void_p)
                    assert pkind[1] == "void*", (name, cp, ct)
                elif pkind[1] is not None:  # a typed pointer names the same base type or struct
                    assert pkind[1] == ckind[1], (name, cp, ct)
            else:
                assert pkind == ckind, (name, cp, ct)
        rk = _c_kind(ret)
        if rk == ("ptr", "char"):
            import ctypes
            assert fn.restype is ctypes.c_char_p, name
        else:
            assert _ctypes_kind(fn.restype) == rk, (name, ret, fn.restype)
