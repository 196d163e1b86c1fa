"""The product path has no CPU fallback and never touches the oracle: no
module of the package imports it, and without libjsvd.so the binding
raises instead of computing anything."""
import ast
import glob
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2202_08361_gb300")


def test_package_never_imports_the_oracle():
    offenders = []
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        tree = ast.parse(open(path).read(), filename=path)
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom) and node.module:
                names = [node.module]
            if any(n == "oracle" or n.startswith("oracle.") for n in names):
                offenders.append(os.path.relpath(path, ROOT))
    assert not offenders, offenders


def test_missing_library_raises():
    code = (
        "from paper_2202_08361_gb300 import build, _native\n"
        "build.LIB = '/nonexistent/libjsvd.so'\n"
        "import paper_2202_08361_gb300 as J\n"
        "try:\n"
        "    J.version()\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    print('no error')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert "raised:" in r.stdout and "not built" in r.stdout, r.stdout + r.stderr
