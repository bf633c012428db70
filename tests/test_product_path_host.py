"""The product path and the oracle stay apart, and the product has no CPU fallback
(CPU only, static checks plus one load attempt):

- the binding raises when libscalefree.so is missing instead of computing anything;
- no module of the package imports the oracle, and the CUDA sources name no oracle
  file;
- the oracle imports nothing from the package;
- bench.py reaches the oracle only inside its CPU-baseline / reference sample
  function.
"""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2601_20758_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(d):
    for base, _, files in os.walk(d):
        if "_build" in base or "__pycache__" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def _imported_modules(path):
    with open(path) as f:
        tree = ast.parse(f.read(), filename=path)
    mods = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods += [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            mods.append(node.module)
    return mods


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2601_20758_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libscalefree.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
    with pytest.raises(RuntimeError, match="not built"):
        _lib.make_params()


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        bad = [m for m in _imported_modules(path) if m == "oracle" or m.startswith("oracle.")]
        assert not bad, f"{path} imports {bad}"
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        with open(os.path.join(csrc, f)) as fh:
            src = fh.read()
        assert "sf_oracle" not in src and "liboracle" not in src, f


def test_oracle_imports_nothing_from_the_package():
    for path in _py_files(ORACLE):
        bad = [m for m in _imported_modules(path) if m.startswith("paper_2601_20758_gb300")]
        assert not bad, f"{path} imports {bad}"


def test_bench_reaches_the_oracle_only_in_its_sample_leg():
    path = os.path.join(ROOT, "bench.py")
    with open(path) as f:
        tree = ast.parse(f.read(), filename=path)
    owners = []
    for fn in ast.walk(tree):
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    owners.append(fn.name)
                if isinstance(node, ast.ImportFrom) and node.level == 0 and node.module == "oracle":
                    owners.append(fn.name)
    top = [n for n in tree.body
           if (isinstance(n, ast.Import) and any(a.name == "oracle" for a in n.names))
           or (isinstance(n, ast.ImportFrom) and n.module == "oracle")]
    assert not top, "bench.py imports the oracle at module level"
    assert owners == ["oracle_sample"], owners
