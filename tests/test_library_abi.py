"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/pc.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pc_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2306_07212_gb300 import buildlib
    return buildlib.build()


def test_library_exports_every_declared_symbol(lib_path):
    declared = _declared()
    assert {"pc_create", "pc_extract", "pc_vertices", "pc_edges", "pc_signvectors", "pc_backward"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pc_[a-z_0-9]+)\b", out))
    assert declared <= exported, f"missing: {declared - exported}"
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert getattr(lib, name)


def test_binding_lists_every_declared_symbol():
    from paper_2306_07212_gb300 import binding
    assert _declared() <= set(binding.EXPORTS) | {"pc_alloc_fn", "pc_free_fn"}


def test_library_targets_sm_103a(lib_path):
    from paper_2306_07212_gb300 import buildlib
    assert "arch=compute_103a,code=sm_103a" in " ".join(buildlib.ARCH)


def test_default_options_without_gpu(lib_path):
    from paper_2306_07212_gb300 import binding
    lib = binding.load_library()
    o = binding.Options()
    lib.pc_default_options(ctypes.byref(o))
    assert o.precision == 1 and o.exec == 0 and o.filter_kappa == 12.0 and o.polish == -1 and o.gemm == 0
