"""Static checks of the separation between the product path and its test
infrastructure: the CUDA library and its binding never reach the oracle,
the oracle and the input generator never reach the library, the
benchmark touches the oracle only in its CPU legs."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2205_03251_gb300")


def _files(*patterns):
    out = []
    for p in patterns:
        out += glob.glob(os.path.join(ROOT, p), recursive=True)
    return sorted(f for f in out if "__pycache__" not in f)


def test_product_never_reaches_the_oracle():
    for f in _files("paper_2205_03251_gb300/**/*.py", "paper_2205_03251_gb300/csrc/*", "include/*.h"):
        assert "oracle" not in open(f, errors="replace").read(), f


def test_oracle_and_generator_never_reach_the_library():
    for f in _files("oracle/*.py", "oracle/*.c", "synth/*.py", "synth/*.c"):
        src = open(f).read()
        assert "paper_2205_03251_gb300" not in src and "gpfdp" not in src, f


def test_benchmark_uses_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, (ast.Import, ast.ImportFrom)):
                    names = [a.name for a in node.names] + [getattr(node, "module", None) or ""]
                    if any(n.split(".")[0] == "oracle" for n in names):
                        users.add(fn.name)
    assert users and users <= {"cpu_baseline", "reference_units", "run_reference"}, users
    for node in tree.body:                                   # no module-level import of it
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            assert all(a.name.split(".")[0] != "oracle" for a in node.names)

