"""The oracle and the library stay apart (CPU only, static).

The library (Python package and CUDA sources) never imports, includes or runs anything of
the oracle, so no product path can route through the CPU oracle.  The oracle includes
nothing of the library; its only inputs from the package are the arrays that the seeded
scene generators build.  bench.py reaches the oracle only inside its CPU-baseline and
reference legs.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2409_16385_gb300")
ORC = os.path.join(ROOT, "oracle")


def _py_files(d):
    for dirpath, dirnames, files in os.walk(d):
        dirnames[:] = [x for x in dirnames if x not in ("__pycache__", "_build")]
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def _imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield ("." * node.level) + (node.module or "")
        elif isinstance(node, ast.Call) and getattr(node.func, "attr", "") == "import_module":
            if node.args and isinstance(node.args[0], ast.Constant):
                yield str(node.args[0].value)


def test_library_never_imports_the_oracle():
    for path in _py_files(PKG):
        for m in _imported_modules(path):
            assert m.split(".")[0] != "oracle", f"{path} imports {m}"
        text = open(path).read()
        assert "liboracle" not in text and "oracle.cpp" not in text, path


def test_cuda_sources_include_nothing_of_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h", ".cpp", ".hpp")):
            for inc in re.findall(r'#include\s+"([^"]+)"', open(os.path.join(csrc, f)).read()):
                assert "oracle" not in inc and os.path.exists(os.path.join(csrc, inc)) or \
                    os.path.exists(os.path.join(ROOT, "include", os.path.basename(inc))), (f, inc)
                assert not os.path.exists(os.path.join(ORC, os.path.basename(inc))), (f, inc)


def test_oracle_includes_and_imports_nothing_of_the_library():
    for f in os.listdir(ORC):
        p = os.path.join(ORC, f)
        if f.endswith((".cpp", ".hpp", ".h")):
            for inc in re.findall(r'#include\s+"([^"]+)"', open(p).read()):
                assert os.path.exists(os.path.join(ORC, inc)), (f, inc)
    for path in _py_files(ORC):
        for m in _imported_modules(path):
            assert not m.startswith("paper_2409_16385_gb300"), f"{path} imports {m}"


def test_bench_reaches_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"oracle_sample", "run_reference", "batched_oracle_sample", "cpu_baseline", "cpu_stage_baseline",
               "cpu_enumeration", "reference_list"}
    for node in tree.body:
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            names = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
            assert all(n.split(".")[0] != "oracle" for n in names), "bench.py imports the oracle at module level"

    def oracle_imports(node):
        for sub in ast.walk(node):
            if isinstance(sub, (ast.Import, ast.ImportFrom)):
                names = [a.name for a in sub.names] if isinstance(sub, ast.Import) else [sub.module or ""]
                if any(n.split(".")[0] == "oracle" for n in names):
                    yield sub

    users = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.FunctionDef) and any(True for _ in oracle_imports(node)):
            users.add(node.name)
    # the GPU arm imports it only in its CPU-baseline branch, after the timed region
    if "run_ours" in users:
        fn = next(n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name == "run_ours")
        inside = set()
        for sub in ast.walk(fn):
            if isinstance(sub, ast.If) and "no_cpu_baseline" in ast.unparse(sub.test):
                inside |= {id(i) for i in oracle_imports(sub)}
        assert all(id(i) in inside for i in oracle_imports(fn))
        users.discard("run_ours")
    assert users and users <= allowed, users
