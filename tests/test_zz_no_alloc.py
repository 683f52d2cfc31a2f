"""GPU test of pc_extract_noalloc, the allocation-free extraction entry point.

Callers that cannot allocate device memory while they run (inside a memory
pool or allocator callback, on real-time paths that forbid cudaMalloc, or
under a fixed memory reservation) call it with their own output arrays; all
other working memory is a fixed static device array inside the library.

The test calls it through the C ABI on several networks in a row, so later
calls run on the scratch contents that earlier calls left behind, and checks
every result against pc_extract's and the FP64 oracle's: identical sign
vectors and edge sets, coordinates within 1e-6 of the box diameter (the
tolerance of the parity tests).  It also runs a call after one that ran out
of capacity, and checks that a misaligned edge capacity is rejected.  This
file runs last (tests/conftest.py orders it after every other module).
"""
import ctypes

import numpy as np
import pytest

from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu

PRECISION = {"fp32": 0, "mixed": 1, "fp64": 2}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor, load_library
    return torch, Extractor, load_library()


def _noalloc(torch, lib, net, box, precision, cap_v, cap_e, expect=0):
    D = net.D
    P = 2 * D + net.n_neurons
    S = (P + 31) // 32
    X = torch.full((D, cap_v), float("nan"), dtype=torch.float64, device="cuda")
    E = torch.full((2, cap_e), -1, dtype=torch.int32, device="cuda")
    SIG = torch.zeros((S, cap_v), dtype=torch.int64, device="cuda")
    widths = np.ascontiguousarray(net.widths, np.int32)
    params = np.ascontiguousarray(net.flat_params(), np.float64)
    lo = np.ascontiguousarray(box.lo, np.float64)
    hi = np.ascontiguousarray(box.hi, np.float64)
    nv, ne = ctypes.c_int64(-1), ctypes.c_int64(-1)
    st = lib.pc_extract_noalloc(net.L, widths.ctypes.data, params.ctypes.data, lo.ctypes.data, hi.ctypes.data,
                                PRECISION[precision], X.data_ptr(), E.data_ptr(), SIG.data_ptr(), cap_v, cap_e,
                                ctypes.byref(nv), ctypes.byref(ne), torch.cuda.current_stream().cuda_stream)
    assert st == expect, f"pc_extract_noalloc returned {st}"
    if st != 0:
        return None
    nv, ne = nv.value, ne.value
    Xh = X[:, :nv].cpu().numpy().T.copy()
    Eh = E[:, :ne].cpu().numpy().T.copy()
    Sh = SIG[:, :nv].cpu().numpy().view(np.uint64)
    return Xh, unpack_codes(Sh, P), Eh


def _reference(Extractor, net, box, precision):
    with Extractor(precision=precision) as ex:
        ex.extract(net, box)
        c = ex.counts()
        return ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges()


def _oracle(net, box):
    import oracle
    r = oracle.extract(net, box)
    assert r.status == 0, r.error
    return r.X, r.S, r.E


@pytest.mark.parametrize("precision", ["mixed", "fp64", "fp32"])
def test_noalloc_matches_extract_on_consecutive_calls(env, precision):
    torch, Extractor, lib = env
    cases = [wl.small_d2(),
             (wl.he_normal_mlp([3, 16, 16, 1], seed=1000), wl.Box.cube(3)),
             wl.small_d2()]
    for net, box in cases:
        got = _noalloc(torch, lib, net, box, precision, cap_v=16384, cap_e=65536)
        ref = _reference(Extractor, net, box, precision)
        tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
        assert_same_complex(got, ref, coord_tol=tol, what=f"noalloc {net.widths} {precision}")
        if precision != "fp32":  # FP32 decisions without the filter may differ from FP64 ones
            assert_same_complex(got, _oracle(net, box), coord_tol=tol, what=f"noalloc vs oracle {net.widths}")


def test_noalloc_after_a_call_that_ran_out_of_capacity(env):
    """A call that outgrows the caller's capacities stops with PC_ERR_OOM and
    leaves its partial state in the shared scratch; the next call must still
    give pc_extract's result."""
    torch, Extractor, lib = env
    net, box = wl.he_normal_mlp([3, 16, 16, 1], seed=1000), wl.Box.cube(3)
    assert _noalloc(torch, lib, net, box, "mixed", cap_v=64, cap_e=4096, expect=2) is None
    assert _noalloc(torch, lib, net, box, "mixed", cap_v=16384, cap_e=256, expect=2) is None
    got = _noalloc(torch, lib, net, box, "mixed", cap_v=16384, cap_e=65536)
    tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    assert_same_complex(got, _reference(Extractor, net, box, "mixed"), coord_tol=tol, what="noalloc after OOM")


def test_noalloc_rejects_a_misaligned_edge_capacity(env):
    """The second endpoint row starts at E + cap_e and is read with 16-byte
    loads, so cap_e must be a multiple of 4: checked on the host, no kernel
    runs."""
    torch, Extractor, lib = env
    net, box = wl.small_d2()
    assert _noalloc(torch, lib, net, box, "mixed", cap_v=1024, cap_e=4099, expect=1) is None
    got = _noalloc(torch, lib, net, box, "mixed", cap_v=1024, cap_e=4100)
    tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    assert_same_complex(got, _oracle(net, box), coord_tol=tol, what="noalloc cap_e 4100")


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, Extractor, lib = env
    net, box = wl.small_d2()
    with pytest.raises(AssertionError, match="returned 6"):
        _noalloc(torch, lib, net, box, "mixed", cap_v=1 << 20, cap_e=65536)
    wide = wl.he_normal_mlp([2, 64, 1], seed=0)
    with pytest.raises(AssertionError, match="returned 6"):
        _noalloc(torch, lib, wide, box, "mixed", cap_v=1024, cap_e=4096)
