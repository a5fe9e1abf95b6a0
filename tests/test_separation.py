"""The oracle and the CUDA path share no code (no GPU needed).

* Nothing in the package (Python binding, C++ runtime, CUDA kernels) or in include/
  imports or includes the oracle.
* The oracle never loads the package, its library or its sources.
* The shared input module `synth` imports neither side.
* bench.py and __graft_entry__.py import the oracle only inside the functions allowed to
  use it: the CPU-baseline and reference legs of the benchmark, and the smoke check.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(sub, exts):
    out = []
    for d, _, names in os.walk(os.path.join(ROOT, sub)):
        if "__pycache__" in d:
            continue
        out += [os.path.join(d, n) for n in names if n.endswith(exts)]
    return out


def _imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    mods = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods += [(a.name.split(".")[0], node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.append((node.module.split(".")[0], node))
    return tree, mods


def test_product_never_imports_the_oracle():
    for path in _files("paper_1311_1646_gb300", (".py",)):
        _, mods = _imported_modules(path)
        assert "oracle" not in [m for m, _ in mods], path
    for path in _files("paper_1311_1646_gb300", (".cpp", ".cu", ".h")) + _files("include", (".h",)):
        src = open(path).read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', src), path


def test_oracle_never_loads_the_product():
    for path in _files("oracle", (".py",)):
        src = open(path).read()
        _, mods = _imported_modules(path)
        names = [m for m, _ in mods]
        assert "paper_1311_1646_gb300" not in names and "ctypes" not in names and "torch" not in names, path
        assert "liblrt" not in src and "csrc" not in src, path


def test_inputs_module_imports_neither_side():
    for path in _files("synth", (".py",)):
        _, mods = _imported_modules(path)
        names = [m for m, _ in mods]
        assert "oracle" not in names and "paper_1311_1646_gb300" not in names, path


def _oracle_imports_by_function(path):
    tree = ast.parse(open(path).read(), path)
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.ImportFrom) and child.module and child.module.split(".")[0] == "oracle":
                found.append(func)
            elif isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append(func)
            visit(child, f)
    visit(tree, None)
    return found


def test_oracle_is_imported_only_by_the_allowed_legs():
    bench = _oracle_imports_by_function(os.path.join(ROOT, "bench.py"))
    assert bench and set(bench) <= {"_oracle_setup", "cpu_baseline", "cpu_baseline_child",
                                     "_child_sigma", "run_reference"}, bench
    entry = _oracle_imports_by_function(os.path.join(ROOT, "__graft_entry__.py"))
    assert entry and set(entry) <= {"smoke"}, entry
