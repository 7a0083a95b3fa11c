"""Static checks of the separation rules (CPU): the library's Python layer never imports the
oracle, the oracle never imports the library, and the input generators import neither; the
binding raises instead of falling back when the compiled library is missing."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                out.add(node.module.split(".")[0])
    return out


def _py_files(folder):
    d = os.path.join(ROOT, folder)
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_product_does_not_import_the_oracle():
    for f in _py_files("paper_1603_06855_gb300"):
        assert not (_imports(f) & {"oracle", "workloads"}), f


def test_oracle_does_not_import_the_product():
    for f in _py_files("oracle"):
        assert "paper_1603_06855_gb300" not in _imports(f), f


def test_inputs_import_neither():
    for f in _py_files("workloads"):
        assert not (_imports(f) & {"oracle", "paper_1603_06855_gb300"}), f


def test_oracle_is_plain_python():
    """The oracle holds no compiled code and does not load shared libraries."""
    for f in _py_files("oracle"):
        assert not (_imports(f) & {"ctypes", "torch", "cffi"}), f
    assert not [f for f in os.listdir(os.path.join(ROOT, "oracle")) if f.endswith((".so", ".c", ".cu", ".cpp"))]


def test_binding_raises_without_the_library(tmp_path):
    from paper_1603_06855_gb300 import binding as B
    saved = B._lib
    B._lib = None
    try:
        with pytest.raises(OSError):
            B.load(str(tmp_path / "missing.so"))
    finally:
        B._lib = saved
