"""The product path and the oracle share no code (checked on the host).

Nothing in the package, the C ABI header or the input generators imports,
includes, links or loads anything under oracle/; the oracle's sources do not
include the library's headers; and the package's binding loads only its own
in-tree library."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2104_05372_b300")


def _files(top, exts):
    for base, _, names in os.walk(top):
        if "__pycache__" in base or "_build" in base:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(base, n)


def test_product_sources_do_not_use_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle)|liboracle", re.M)
    offenders = []
    for top in (PKG, os.path.join(ROOT, "include"), os.path.join(ROOT, "synth")):
        for p in _files(top, (".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
            if pat.search(open(p, encoding="utf-8", errors="replace").read()):
                offenders.append(os.path.relpath(p, ROOT))
    assert offenders == []


def test_oracle_sources_do_not_use_the_library():
    pat = re.compile(r"#\s*include\s*[<\"](gpa\.h|[^>\"]*csrc)|paper_2104_05372_b300|libgpa")
    for p in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        assert not pat.search(open(p, encoding="utf-8", errors="replace").read()), os.path.relpath(p, ROOT)


def test_binding_loads_its_in_tree_library():
    src = open(os.path.join(PKG, "_lib.py"), encoding="utf-8").read()
    assert "libgpa.so" in src and "oracle" not in src
