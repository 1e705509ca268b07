"""The CUDA path and the oracle share no code, and the product path never
reaches the oracle.

Static checks of the sources: the package and the CUDA library name no
oracle module, file or symbol; the oracle includes no header of the
library and imports nothing of the package except the seeded input
generators (which hold none of the method's arithmetic); synth imports
neither side.
"""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2512_11606_gb300")


def py_imports(path):
    tree = ast.parse(open(path, encoding="utf-8").read(), path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mods.add(("." * node.level) + (node.module or ""))
    return mods


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        mods = py_imports(path)
        assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), path


def test_cuda_sources_name_nothing_of_the_oracle():
    srcs = glob.glob(os.path.join(PKG, "csrc", "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert srcs
    for path in srcs:
        text = open(path, encoding="utf-8").read()
        assert not re.search(r"ahpp_oracle|\bog_[a-z]+\(|oracle/", text), path


def test_oracle_uses_no_library_code():
    c_src = open(os.path.join(ROOT, "oracle", "ahpp_oracle.c"), encoding="utf-8").read()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', c_src)
    assert all(not inc.startswith("ahpp") or inc.startswith("ahpp_oracle") for inc in includes), includes
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for m in py_imports(path):
            if m.startswith("paper_2512_11606_gb300"):
                assert m == "paper_2512_11606_gb300.synth" or m == "paper_2512_11606_gb300", (path, m)


def test_input_generators_import_neither_side():
    mods = py_imports(os.path.join(PKG, "synth.py"))
    for m in mods:
        assert not m.startswith("oracle") and "ahpp" not in m and "build" not in m, m
