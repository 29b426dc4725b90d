"""The CUDA path and the oracle share no code, and the product path never
reaches the oracle: no import or #include crosses between them, the two
shared libraries neither link nor export each other's symbols, importing the
package loads no oracle module, and the seeded input module depends on
neither.  CPU only (the libraries are built, not run)."""
import ast
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2609_12476_gb300")
ORACLE = os.path.join(ROOT, "oracle")
SYNTH = os.path.join(ROOT, "srs_synth")


def _py_files(d):
    for dirpath, _, names in os.walk(d):
        if "__pycache__" in dirpath:
            continue
        for n in names:
            if n.endswith(".py"):
                yield os.path.join(dirpath, n)


def _imported_roots(path):
    tree = ast.parse(open(path).read(), path)
    roots = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            roots.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            roots.add(node.module.split(".")[0])
    return roots


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), re.M)


def test_package_never_imports_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imported_roots(f), f


def test_oracle_never_imports_the_package():
    for f in _py_files(ORACLE):
        assert "paper_2609_12476_gb300" not in _imported_roots(f), f


def test_input_module_depends_on_neither_side():
    for f in _py_files(SYNTH):
        roots = _imported_roots(f)
        assert "oracle" not in roots and "paper_2609_12476_gb300" not in roots, f


def test_no_include_crosses_between_the_sides():
    csrc = os.path.join(PKG, "csrc")
    for n in os.listdir(csrc):
        for inc in _includes(os.path.join(csrc, n)):
            assert "oracle" not in inc, (n, inc)
    for n in os.listdir(ORACLE):
        if n.endswith((".c", ".h")):
            for inc in _includes(os.path.join(ORACLE, n)):
                assert "srs" not in inc and "csrc" not in inc and "include/" not in inc, (n, inc)


def _dynamic_symbols(so):
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    return {line.split()[-1] for line in out.splitlines() if line.strip()}


def _needed(so):
    out = subprocess.run(["readelf", "-d", so], capture_output=True, text=True, check=True).stdout
    return re.findall(r"\(NEEDED\)\s+Shared library: \[([^\]]+)\]", out)


def test_libraries_neither_link_nor_export_each_other():
    if not (shutil.which("nm") and shutil.which("readelf")):
        pytest.skip("binutils not installed")
    from oracle import build as obuild
    from paper_2609_12476_gb300 import build as libbuild
    srs_so = libbuild.build()
    orc_so = obuild.build()
    srs_syms, orc_syms = _dynamic_symbols(srs_so), _dynamic_symbols(orc_so)
    assert not any(s.startswith("orc_") for s in srs_syms)
    assert not any(s.startswith("srs_") for s in orc_syms)
    assert not any("oracle" in n for n in _needed(srs_so))
    assert not any("srs" in n for n in _needed(orc_so))


def test_importing_the_package_loads_no_oracle_module():
    code = ("import sys; import paper_2609_12476_gb300 as p; p.nsigma_threshold(3, 1e-3); "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "print(bad); sys.exit(1 if bad else 0)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
