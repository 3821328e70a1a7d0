"""The oracle and the CUDA path share no code: the product package never imports the oracle, the
oracle imports neither the product nor the input generators, and the generators (the one module
both sides read) import neither.  The product also has no fallback: without its compiled library
it raises instead of computing anything."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2201_10062_gb300"


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def _py_files(d):
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_product_never_imports_the_oracle():
    for path in _py_files(os.path.join(ROOT, PKG)):
        assert "oracle" not in _imports(path), path
    csrc = os.path.join(ROOT, PKG, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f), errors="replace").read()
        assert not re.search(r'#include\s*[<"][^>"]*oracle', text), f


def test_oracle_imports_neither_the_product_nor_the_generators():
    for path in _py_files(os.path.join(ROOT, "oracle")):
        imp = _imports(path)
        assert PKG not in imp and "workloads" not in imp, (path, imp)


def test_generators_import_neither_side():
    for path in _py_files(os.path.join(ROOT, "workloads")):
        imp = _imports(path)
        assert PKG not in imp and "oracle" not in imp, (path, imp)


def test_no_fallback_without_the_library(tmp_path):
    """load_library refuses a missing library: there is no CPU path to fall back on."""
    import paper_2201_10062_gb300 as P

    saved = P._lib
    P._lib = None
    try:
        with pytest.raises(ImportError):
            P.load_library(str(tmp_path / "missing.so"))
    finally:
        P._lib = saved
