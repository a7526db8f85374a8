"""The oracle and the CUDA path share no code: nothing in the package imports,
includes or loads the oracle, and the oracle imports nothing from the package.
Only the tests, the smoke check and the benchmark's CPU-baseline and reference
legs may use the oracle."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1701_03891_gb300")


def _py_imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def test_package_never_uses_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        assert "oracle" not in _py_imports(path), path
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        src = open(path).read()
        assert not re.search(r'#include\s*["<][^">]*oracle', src), path
        assert "liboracle" not in src, path


def test_oracle_imports_nothing_from_the_package():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_1701_03891_gb300" not in _py_imports(path), path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.c")):
        src = open(path).read()
        includes = re.findall(r'#include\s*["<]([^">]+)[">]', src)
        assert all("/" not in inc and not inc.endswith((".cuh", "deepinv.h")) for inc in includes), includes


def test_only_permitted_places_use_the_oracle():
    """Outside tests/ and oracle/, only the smoke check and bench.py's
    CPU-baseline and reference legs import it (and build(), which compiles the
    oracle's C source without running it)."""
    users = {}
    for path in glob.glob(os.path.join(ROOT, "*.py")):
        tree = ast.parse(open(path).read())
        for fn in ast.walk(tree):
            if isinstance(fn, ast.FunctionDef):
                for node in ast.walk(fn):
                    if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                        users.setdefault(os.path.basename(path), set()).add(fn.name)
        top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
        assert not any(isinstance(n, ast.Import) and any(a.name == "oracle" for a in n.names) for n in top), path
    assert users == {"__graft_entry__.py": {"build", "smoke"}, "bench.py": {"cpu_baseline", "run_reference"}}, users
