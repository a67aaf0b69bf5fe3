"""The oracle and the CUDA path stay apart: the product package never
imports the oracle, the oracle never imports the product, the benchmark
touches the oracle only in its CPU-baseline sample, and a missing CUDA library
is an error, not a fallback."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    """(module name, enclosing function or None) of every import in a file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, fn):
        for ch in ast.iter_child_nodes(node):
            f = ch.name if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(ch, ast.Import):
                out.extend((a.name, f) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom) and ch.level == 0 and ch.module:
                out.append((ch.module, f))
            visit(ch, f)
    visit(tree, None)
    return out


def _py_files(d):
    for base, _, files in os.walk(os.path.join(ROOT, d)):
        if "__pycache__" in base or "_build" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_product_package_never_imports_the_oracle():
    for path in _py_files("paper_2601_23002_gb300"):
        for mod, _ in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)


def test_oracle_never_imports_the_product():
    for path in _py_files("oracle"):
        for mod, _ in _imports(path):
            assert mod.split(".")[0] not in ("paper_2601_23002_gb300", "bench"), (path, mod)


def test_benchmark_uses_the_oracle_only_for_its_cpu_baseline():
    uses = [(m, f) for m, f in _imports(os.path.join(ROOT, "bench.py")) if m.split(".")[0] == "oracle"]
    assert uses, "the CPU baseline times the oracle"
    assert {f for _, f in uses} <= {"oracle_sample"}, uses


def test_missing_cuda_library_is_an_error_not_a_fallback(tmp_path, monkeypatch):
    from paper_2601_23002_gb300 import _lib, build
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(build, "build", lambda *a, **k: None)     # nothing gets built
    with pytest.raises(OSError):
        _lib.load(str(tmp_path / "libofdft_gb300.so"))
