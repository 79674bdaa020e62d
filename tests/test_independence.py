"""The oracle and the CUDA path share no code (CPU only, by parsing the sources): the package and
the input generators never import the oracle, the oracle never imports the package, the native
sources include nothing from it, and bench.py reaches the oracle only from its reference arm and
CPU-baseline helpers."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def py_files(rel):
    out = []
    for d, dirs, files in os.walk(os.path.join(ROOT, rel)):
        dirs[:] = [x for x in dirs if not x.startswith(("_build", "__pycache__"))]
        out += [os.path.join(d, f) for f in files if f.endswith(".py")]
    return out


def imported_modules(tree):
    """(top-level package of every import, enclosing function name or None)."""
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name.split(".")[0], fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.level == 0 and child.module:
                out.append((child.module.split(".")[0], fn))
            visit(child, name)

    visit(tree, None)
    return out


def test_package_and_generators_never_import_the_oracle():
    files = py_files("paper_2507_01631_b300") + py_files("synth")
    assert len(files) > 5
    for f in files:
        mods = imported_modules(ast.parse(open(f).read()))
        assert "oracle" not in [m for m, _ in mods], f


def test_oracle_never_imports_the_package():
    for f in py_files("oracle"):
        mods = [m for m, _ in imported_modules(ast.parse(open(f).read()))]
        assert "paper_2507_01631_b300" not in mods and "bench" not in mods, f


def test_native_sources_include_nothing_from_the_oracle():
    for d in ("paper_2507_01631_b300/csrc", "include"):
        for f in os.listdir(os.path.join(ROOT, d)):
            if f.endswith((".cu", ".cuh", ".h")):
                for line in open(os.path.join(ROOT, d, f)):
                    assert not (line.lstrip().startswith("#include") and "oracle" in line), (f, line)


def test_bench_reaches_the_oracle_only_from_its_reference_helpers():
    mods = imported_modules(ast.parse(open(os.path.join(ROOT, "bench.py")).read()))
    users = {fn for m, fn in mods if m == "oracle"}
    assert users and users <= {"oracle_sample", "oracle_grid_params", "run_reference"}, users
