"""The product path has no fallback: without the CUDA library every call of
the binding raises, and nothing in the package reaches the oracle."""

import ast
import glob
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2306_06983_gb300")


def test_missing_library_fails_loudly():
    """A fresh interpreter whose binding points at a library that does not
    exist: the first call that needs it raises RuntimeError naming the
    missing build (no CPU path is tried)."""
    code = (
        "import paper_2306_06983_gb300.nlbm as N\n"
        "from paper_2306_06983_gb300 import workloads as W\n"
        "N.load_library.__defaults__ = ('/nonexistent/libnlbm.so',)\n"
        "p, _ = W.droplets_64('B')\n"
        "try:\n"
        "    N.nlbm_workspace_bytes(p)\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    print('no error')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "raised:" in r.stdout and "not built" in r.stdout, r.stdout


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            else:
                continue
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)


def test_cuda_sources_never_include_the_oracle():
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        for line in open(path):
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line, (path, line)
