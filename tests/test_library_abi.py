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


@pytest.mark.parametrize("variant", ["libpc.so", "libpc_d10.so"])
def test_library_exports_every_declared_symbol(lib_path, variant):
    declared = _declared()
    assert {"pc_create", "pc_extract", "pc_vertices", "pc_edges", "pc_signvectors", "pc_backward"} <= declared
    path = os.path.join(os.path.dirname(lib_path), variant)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pc_[a-z_0-9]+)\b", out))
    assert declared <= exported, f"missing: {declared - exported}"
    lib = ctypes.CDLL(path)
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


def test_memory_estimate_covers_the_oracle_complex(lib_path):
    """The serving admission estimate (pc_estimate_bytes, host-only) covers
    the device bytes of the complex the oracle extracts for random nets of the
    serving mix (coordinates, two value rows per vertex, sign words, edges,
    staging), with room for one capacity doubling."""
    import numpy as np
    import oracle
    from paper_2306_07212_gb300 import workloads as wl
    from paper_2306_07212_gb300.binding import estimate_bytes
    for D, depth, width, seed in [(2, 2, 16, 0), (2, 4, 32, 1), (3, 2, 16, 2), (3, 3, 16, 3), (4, 2, 8, 4),
                                  (2, 6, 16, 5), (3, 2, 32, 6)]:
        net = wl.he_normal_mlp([D] + [width] * depth + [1], seed=seed)
        r = oracle.extract(net, wl.Box.cube(D))
        S = (2 * D + net.n_neurons + 31) // 32
        need = r.nV * (8 * D + 2 * 4 * width + 8 + 8 * S) + len(r.E) * (8 + 16)
        est = estimate_bytes(net)
        assert est >= 2 * need, (D, depth, width, est, need)
        assert est < 1e12
    # monotone in width and depth
    small = estimate_bytes(wl.he_normal_mlp([3, 16, 16, 1], seed=0))
    assert estimate_bytes(wl.he_normal_mlp([3, 32, 16, 1], seed=0)) > small
    assert estimate_bytes(wl.he_normal_mlp([3, 16, 16, 16, 1], seed=0)) > small


def test_header_is_plain_c_and_host_calls_work(lib_path, tmp_path):
    """include/pc.h compiles as strict C99 (-Wall -Wextra -Werror -pedantic);
    a C program links libpc.so and calls the entry points that need no GPU."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_host")
    src = os.path.join(ROOT, "tests", "c", "abi_host.c")
    libdir = os.path.dirname(lib_path)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I" + os.path.join(ROOT, "include"),
                        src, "-L" + libdir, "-lpc", "-Wl,-rpath," + libdir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")


def test_ctypes_structures_match_the_header(tmp_path):
    """Every field of pc_options, pc_server_options and pc_result sits at the
    same offset in the binding's ctypes structures as in the C header, and
    the structures have the same size."""
    import shutil
    from paper_2306_07212_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "layout")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "layout.c"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    classes = {"pc_options": binding.Options, "pc_server_options": binding.ServerOptions,
               "pc_result": binding.Result}
    seen = {k: set() for k in classes}
    for line in filter(None, out):
        struct, field, value = line.split()
        cls = classes[struct]
        if field == "sizeof":
            assert ctypes.sizeof(cls) == int(value), struct
        else:
            assert getattr(cls, field).offset == int(value), (struct, field)
            seen[struct].add(field)
    for struct, cls in classes.items():
        assert seen[struct] == {f for f, _ in cls._fields_}, struct


def test_binding_argtypes_match_the_header_arity(lib_path):
    """Every function of include/pc.h has ctypes argtypes in the binding with
    as many parameters as the declaration."""
    from paper_2306_07212_gb300 import binding
    src = open(os.path.join(ROOT, "include", "pc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"\b(pc_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src)
    lib = binding.load_library()
    checked = 0
    for name, params in decls:
        params = " ".join(params.split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None, f"{name} has no argtypes in the binding"
        assert len(argtypes) == n, (name, len(argtypes), n)
        checked += 1
    assert checked >= 30
