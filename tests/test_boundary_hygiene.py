"""Structure of the code base (CPU only, by reading the sources): the product path never reaches
the oracle, the oracle never reaches the product path, and the seeded input generators, the one
module both sides share, import neither. The benchmark touches the oracle only in the class that
runs an oracle chain for its CPU baselines and reference arm, and the package entry only in
smoke()."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2511_06407_b300"


def _imports(path):
    """[(top-level module name, enclosing class and function names)] for every import in the file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, funcs):
        for child in ast.iter_child_nodes(node):
            scope = (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)
            f = funcs + [child.name] if isinstance(child, scope) else funcs
            if isinstance(child, ast.Import):
                out.extend((a.name.split(".")[0], tuple(funcs)) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                if child.level:  # relative import inside a package
                    pkg = os.path.basename(os.path.dirname(path))
                    out.append((pkg, tuple(funcs)))
                else:
                    out.append((child.module.split(".")[0], tuple(funcs)))
            visit(child, f)

    visit(tree, [])
    return out


def test_product_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, PKG, "*.py")):
        mods = {m for m, _ in _imports(path)}
        assert "oracle" not in mods, path


def test_oracle_never_imports_the_product_path():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        mods = {m for m, _ in _imports(path)}
        assert not mods & {PKG, "torch", "ctypes", "bench"}, (path, mods)


def test_input_generators_hold_no_side_of_the_method():
    mods = {m for m, _ in _imports(os.path.join(ROOT, PKG, "workloads.py"))}
    assert mods <= {"numpy", "math"}, mods


def test_benchmark_and_entry_touch_the_oracle_only_in_their_baseline_and_smoke_functions():
    for name, allowed in (("bench.py", {"OracleChain"}), ("__graft_entry__.py", {"smoke"})):
        for mod, funcs in _imports(os.path.join(ROOT, name)):
            if mod == "oracle":
                assert funcs and funcs[0] in allowed, (name, funcs)
