"""The oracle and the product path share no code, and the product path has no CPU fallback.

Static checks (no GPU): no module of the package imports the oracle and no CUDA source
includes a file of it; the oracle imports nothing of the package and includes none of its
headers; the only module both sides may use, the seeded input generators, holds no
arithmetic of the method.  And the binding refuses to run when the CUDA library is
missing instead of computing anything itself.
"""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2504_10539_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or os.sep + "_lib" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), flags=re.M)


def test_package_never_imports_or_includes_the_oracle():
    for p in _files(PKG, (".py",)):
        assert "oracle" not in _imported_modules(p), p
    for p in _files(PKG, (".cu", ".cuh", ".h", ".c", ".cpp")):
        for inc in _includes(p):
            assert "oracle" not in inc, (p, inc)


def test_oracle_never_imports_or_includes_the_package():
    for p in _files(ORACLE, (".py",)):
        assert "paper_2504_10539_gb300" not in _imported_modules(p), p
    csrc = {n for n in os.listdir(os.path.join(PKG, "csrc"))}
    headers = {n for n in os.listdir(os.path.join(ROOT, "include"))}
    for p in _files(ORACLE, (".c", ".h")):
        for inc in _includes(p):
            assert os.path.basename(inc) not in csrc | headers, (p, inc)


def test_shared_input_module_holds_no_method_arithmetic():
    """workloads.py draws numbers; the method's functions live on each side separately."""
    src = open(os.path.join(PKG, "workloads.py")).read()
    tree = ast.parse(src)
    names = {n.name for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.ClassDef))}
    for forbidden in ("equilibrium", "collide", "stream", "step", "psi", "force", "density", "metrics",
                      "correct", "mlp_forward", "grad_mag", "init_rho", "init_equilibrium"):
        assert forbidden not in names, forbidden
    assert "import oracle" not in src and "binding" not in _imported_modules(os.path.join(PKG, "workloads.py"))


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2504_10539_gb300 import binding as B
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "missing" / "libpinnlbm.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        B.pl_params_default(8, 8)
