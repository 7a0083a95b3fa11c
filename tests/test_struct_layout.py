"""The ctypes mirrors of the C-ABI structs and constants (binding.py) match include/phononic.h:
a small C program compiled against the header prints sizeof and every field's offsetof, and each
must equal the ctypes size and field offset.  CPU only (gcc); a mismatch would make the binding
read or write the wrong bytes without any error."""
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
