"""The product path never reaches the oracle and has no CPU fallback.

* No module of the package imports ``oracle`` (read statically, and checked
  again after importing every module in a fresh interpreter).
* Without the built library the binding refuses to load instead of
  computing anything on the host.
"""
import ast
import os
import subprocess
import sys

import pytest

from paper_2207_11638_gb300 import binding as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2207_11638_gb300")


def package_modules():
    return sorted(f[:-3] for f in os.listdir(PKG) if f.endswith(".py") and f != "__init__.py")


def test_no_module_of_the_package_imports_the_oracle():
    for name in package_modules() + ["__init__"]:
        tree = ast.parse(open(os.path.join(PKG, name + ".py")).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            else:
                continue
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (name, mods)


def test_importing_the_package_loads_no_oracle_module():
    mods = ", ".join(f"paper_2207_11638_gb300.{m}" for m in package_modules() if m not in ("build",))
    code = (f"import importlib, sys\n"
            f"for m in '{mods}'.split(', '):\n"
            f"    importlib.import_module(m)\n"
            f"bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n"
            f"assert not bad, bad\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]


def test_binding_refuses_to_load_without_the_library(tmp_path):
    with pytest.raises(ImportError, match="is missing"):
        b.load_library(str(tmp_path / "libcdct.so"))
