"""CPU checks that the oracle and the CUDA path stay independent, read from the sources.

* No module of the package imports the oracle, so no product call can route through it.
* The oracle imports nothing of the package and includes no header of the CUDA sources.
* The CUDA sources include no oracle header.
* The library's build names no oracle file.
* bench.py imports the oracle only inside its CPU-baseline and reference-arm functions. The
  timed GPU steps never touch it.
* The seeded input generators, the one module both sides use, import neither side.
"""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2502_08470_gb300")
CSRC = os.path.join(PKG, "csrc")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(tree):
    """(module name, enclosing top-level function or None) for every import in a module."""
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = func
            if func is None and isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)):
                f = child.name
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = child.module or ""
                out.append((mod, f))
                out.extend((f"{mod}.{a.name}" if mod else a.name, f) for a in child.names)
            visit(child, f)

    visit(tree, None)
    return out


def _parse(path):
    with open(path) as fh:
        return ast.parse(fh.read(), filename=path)


def test_the_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        for name, _ in _imports(_parse(path)):
            assert name != "oracle" and not name.startswith("oracle."), (path, name)


def test_the_oracle_uses_nothing_of_the_cuda_path():
    for path in glob.glob(os.path.join(ORACLE, "*.py")):
        for name, _ in _imports(_parse(path)):
            assert not name.startswith("paper_2502_08470_gb300"), (path, name)
    for path in glob.glob(os.path.join(ORACLE, "*.c")) + glob.glob(os.path.join(ORACLE, "*.h")):
        with open(path) as fh:
            for inc in re.findall(r'#include\s+"([^"]+)"', fh.read()):
                assert os.path.exists(os.path.join(ORACLE, inc)), (path, inc)  # its own headers only
                assert "csrc" not in inc and "sigkernel.h" not in inc, (path, inc)


def test_the_cuda_sources_include_no_oracle_file():
    for path in glob.glob(os.path.join(CSRC, "*")):
        if not path.endswith((".cu", ".cuh", ".h")):
            continue
        with open(path) as fh:
            for inc in re.findall(r'#include\s+"([^"]+)"', fh.read()):
                assert "oracle" not in inc, (path, inc)
    with open(os.path.join(PKG, "build.py")) as fh:
        assert "oracle" not in fh.read()


def test_bench_touches_the_oracle_only_in_its_cpu_legs():
    allowed = {"cpu_fwd_bwd", "oracle_samples"}
    for name, func in _imports(_parse(os.path.join(ROOT, "bench.py"))):
        if name == "oracle" or name.startswith("oracle."):
            assert func in allowed, func


def test_the_input_generators_import_neither_side():
    for name, _ in _imports(_parse(os.path.join(PKG, "workloads.py"))):
        assert name.split(".")[0] in {"__future__", "numpy"}, name
