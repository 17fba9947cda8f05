"""The oracle and the CUDA path stay independent (CPU, by reading the code):
no module of the package imports the oracle, the oracle imports neither the
package nor torch nor ctypes (only numpy, scipy's FFT and the standard library), bench.py and the smoke check reach the oracle
only inside the functions allowed to run it, and the binding refuses to run
without the compiled library (no CPU fallback)."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1511_07482_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    """(module name, enclosing top-level function or None) for every import."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, fn):
        for ch in ast.iter_child_nodes(node):
            f = fn
            if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) and fn is None:
                f = ch.name
            if isinstance(ch, ast.Import):
                out.extend((a.name, f) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom):
                out.append(("." * ch.level + (ch.module or ""), f))
            visit(ch, f)

    visit(tree, None)
    return out


def _py_files(d):
    for base, _, files in os.walk(d):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_package_never_imports_the_oracle():
    for p in _py_files(PKG):
        for mod, _ in _imports(p):
            assert not mod.split(".")[0] == "oracle", (p, mod)
    for base, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            src = open(os.path.join(base, f)).read()
            assert "#include \"../../oracle" not in src and "oracle/" not in src, f


def test_oracle_imports_only_the_standard_library_and_numpy():
    # scipy for its FFT only (pocketfft on every host core, the FP64 FFT tier of the oracle)
    allowed = {"numpy", "scipy", "math", "itertools", "__future__", "functools", "typing"}
    for p in _py_files(ORACLE):
        for mod, _ in _imports(p):
            if mod.startswith("."):
                continue
            assert mod.split(".")[0] in allowed, (p, mod)


def test_oracle_reached_only_where_allowed():
    # bench.py: the oracle arm and the cpu_baseline leg's checks (oracle_evals,
    # search_parity), reached from cpu_baseline and run_reference only
    allowed = {os.path.join(ROOT, "bench.py"): {"oracle_evals", "search_parity"},
               os.path.join(ROOT, "__graft_entry__.py"): {"smoke"}}
    for path, fns in allowed.items():
        for mod, fn in _imports(path):
            if mod.split(".")[0] == "oracle":
                assert fn in fns, (path, mod, fn)


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_1511_07482_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError):
        _lib.load(str(tmp_path / "libkdefft.so"))
