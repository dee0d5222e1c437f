"""The oracle and the CUDA path share no code: neither imports or includes the other, and the
product package never reaches the oracle (only the tests, the smoke check and the bench's CPU
legs may)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1112_1071_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield ("." * node.level) + (node.module or "")


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path, errors="replace").read(), flags=re.M)


def test_product_package_never_imports_the_oracle():
    for f in _files(PKG, (".py",)):
        for mod in _imports(f):
            assert not mod.split(".")[0] == "oracle", (f, mod)
    for f in _files(PKG, (".cu", ".cuh", ".h", ".cpp", ".c")):
        for inc in _includes(f):
            assert "oracle" not in inc, (f, inc)


def test_oracle_never_imports_the_product():
    for f in _files(ORACLE, (".py",)):
        for mod in _imports(f):
            root = mod.lstrip(".").split(".")[0]
            assert root not in ("paper_1112_1071_gb300", "torch", "bench"), (f, mod)
    for f in _files(ORACLE, (".c", ".h", ".cpp")):
        for inc in _includes(f):
            assert "csrc" not in inc and "hrt" not in inc, (f, inc)


def test_bench_reaches_the_oracle_only_in_its_cpu_legs():
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path).read(), path)
    for node in tree.body:                                   # no module-level import of the oracle
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            names = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
            assert not any(n.split(".")[0] == "oracle" for n in names)
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                    users.add(fn.name)
                if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                    users.add(fn.name)
    assert users == {"cpu_oracle_rate"}, users
