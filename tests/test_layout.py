"""The oracle and the library stay independent: no product module imports
or loads anything under oracle/, the oracle imports nothing of the package,
and the CUDA sources include nothing of the oracle.  Only the input
generators (synth.py) serve both sides, and the oracle does not use them.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1012_2865_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(d):
    for base, _, files in os.walk(d):
        if "__pycache__" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                names.add(node.module.split(".")[0])
            elif node.level > 0:
                names.add("." + (node.module or ""))
    return names


def test_package_does_not_import_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imports(f), f
        src = open(f).read()
        assert "rt_oracle" not in src and "liboracle" not in src, f


def test_oracle_does_not_import_the_package():
    for f in _py_files(ORACLE):
        imps = _imports(f)
        assert "paper_1012_2865_gb300" not in imps, f
        assert not any(i.startswith(".") and i not in (".", ".timestep") for i in imps), (f, imps)


def test_cuda_sources_include_nothing_of_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        src = open(os.path.join(csrc, f)).read()
        for inc in re.findall(r'#include\s+"([^"]+)"', src):
            assert "oracle" not in inc, (f, inc)
    for f in os.listdir(ORACLE):
        if f.endswith((".c", ".h")):
            src = open(os.path.join(ORACLE, f)).read()
            for inc in re.findall(r'#include\s+"([^"]+)"', src):
                assert not os.path.exists(os.path.join(csrc, os.path.basename(inc))), (f, inc)
