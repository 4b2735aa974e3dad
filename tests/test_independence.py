"""The CUDA path and the oracle stay independent, and the product path has
no CPU fallback:

- no source of the package (Python binding, CUDA kernels, host C++) imports,
  includes, loads or links anything of the oracle;
- the oracle's C source includes only system headers and its wrapper imports
  nothing of the package, so the two share no kernel, helper, table or
  constant generator;
- the one module both sides receive inputs from draws items and imports
  nothing but numpy and the standard library;
- the binding raises, naming the missing library, when the CUDA library is
  absent, instead of computing anything on the host."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2310_14565_gb300")
SOURCE_EXT = (".py", ".cu", ".cuh", ".h", ".hpp", ".cpp", ".c")


def package_sources():
    out = []
    for base, dirs, files in os.walk(PKG):
        dirs[:] = [d for d in dirs if d not in ("__pycache__", "_build")]
        out += [os.path.join(base, f) for f in files if f.endswith(SOURCE_EXT)]
    return sorted(out)


def python_imports(path):
    tree = ast.parse(open(path).read(), path)
    names = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names += [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom):
            names.append(node.module or "")
    return names


def test_package_sources_found():
    names = {os.path.basename(p) for p in package_sources()}
    assert {"__init__.py", "kernels.cu", "pepsi.cu", "host.cpp"} <= names


@pytest.mark.parametrize("path", package_sources(), ids=lambda p: os.path.relpath(p, ROOT))
def test_package_uses_nothing_of_the_oracle(path):
    src = open(path).read()
    if path.endswith(".py"):
        assert not any(n == "oracle" or n.startswith("oracle.") for n in python_imports(path))
        assert not re.search(r"liboracle|oracle[/\\]|pepsi_oracle", src)
    else:
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', src):
            assert "oracle" not in inc, inc
        assert not re.search(r"liboracle|pepsi_oracle|\bor_[a-z0-9_]+\s*\(", src)


def test_oracle_uses_nothing_of_the_package():
    src = open(os.path.join(ROOT, "oracle", "pepsi_oracle.c")).read()
    system = {"math.h", "stdint.h", "stdlib.h", "string.h", "stdio.h", "omp.h", "stddef.h", "limits.h"}
    for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', src):
        assert inc in system, inc
    for name in python_imports(os.path.join(ROOT, "oracle", "__init__.py")):
        assert not name.startswith("paper_2310_14565_gb300"), name


def test_shared_input_module_draws_items_only():
    path = os.path.join(PKG, "workload.py")
    allowed = {"__future__", "dataclasses", "numpy", "typing"}
    assert set(python_imports(path)) <= allowed


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    import paper_2310_14565_gb300 as pepsi

    monkeypatch.setattr(pepsi, "_lib", None)
    monkeypatch.setattr(pepsi, "LIB_PATH", str(tmp_path / "libpepsi_gb300.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pepsi.lib()
