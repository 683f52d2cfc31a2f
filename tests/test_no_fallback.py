"""The product path has no CPU fallback and never touches the oracle: no
module of the package imports it, the CUDA sources share nothing with it, and
loading the binding without the compiled library raises."""
import ast
import glob
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2306_07212_gb300")


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        tree = ast.parse(open(path).read())
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), path


def test_cuda_sources_include_nothing_of_the_oracle():
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        src = open(path).read()
        assert "oracle" not in src.lower(), path


def test_missing_library_raises():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2306_07212_gb300 import binding\n"
            "binding._lib = None\n"
            "try:\n"
            "    binding.load_library('/nonexistent/libpc.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'no CPU fallback' in str(e))\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr


def test_oracle_includes_only_standard_headers():
    src = open(os.path.join(ROOT, "oracle", "oracle.cpp")).read()
    includes = [l.split()[1] for l in src.splitlines() if l.startswith("#include")]
    assert includes and all(i.startswith("<") for i in includes), includes
