"""Failure paths that return a status instead of a result, made without any
GPU fault: every failure here comes from the input, a host-side budget or a
bounded device wait that is made to run out.

* A non-generic network (Section 3.2 assumes that no more than D folded
  hyperplanes meet at a point): the first neuron x + y vanishes exactly at two
  box corners.  Without ``strict`` the extraction succeeds and counts the
  genericity violations; with ``strict`` it returns PC_ERR_DEGENERATE.
* A device-memory budget (``mem_budget_bytes``) too small for the buffers, at
  the first allocation and during capacity growth: PC_ERR_OOM, and the same
  context then extracts a smaller network correctly.
* The persistent kernel's grid barrier with its test switch on waits for an
  arrival that never comes and gives up after a short spin limit:
  PC_ERR_TIMEOUT, repeatably, and the GPU keeps working.
"""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Extractor():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


def _same_as_oracle(ex, net, box, what):
    ref = oracle.extract(net, box)
    assert ref.status == 0, ref.error
    c = ex.counts()
    got = (ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges())
    tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    assert_same_complex(got, (ref.X, ref.S, ref.E), coord_tol=tol, what=what)


def _corner_net():
    """z_1 = x + y is exactly 0 at the corners (1, -1) and (-1, 1)."""
    W = [np.array([[1.0, 1.0], [0.7, -0.4]]), np.array([[0.5, -1.1]])]
    b = [np.array([0.0, 0.13]), np.array([0.05])]
    return wl.Net([2, 2, 1], W, b), wl.Box.cube(2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_generic_network_is_counted_and_strict_rejects_it(Extractor, precision):
    from paper_2306_07212_gb300.binding import PcError
    net, box = _corner_net()
    with Extractor(precision=precision) as ex:
        ex.extract(net, box)
        d = ex.diagnostics()
        assert d["degenerate"] + d["undecided"] > 0, d
    with Extractor(precision=precision, strict=True) as ex:
        with pytest.raises(PcError) as e:
            ex.extract(net, box)
        assert e.value.status == 4, str(e.value)
        assert "genericity" in str(e.value)
        ok, okb = wl.small_d2()
        ex.extract(ok, okb)  # generic: strict passes
        _same_as_oracle(ex, ok, okb, f"strict {precision} after a rejection")


def test_budget_too_small_for_the_first_allocation(Extractor):
    from paper_2306_07212_gb300.binding import PcError
    big = wl.he_normal_mlp([3, 64, 64, 1], seed=3)
    with Extractor(precision="mixed", mem_budget_bytes=8 << 20) as ex:
        with pytest.raises(PcError) as e:
            ex.extract(big, wl.Box.cube(3))
        assert e.value.status == 2, str(e.value)
        net, box = wl.small_d2()
        ex.extract(net, box)
        _same_as_oracle(ex, net, box, "after a failed first allocation")
        assert ex.diagnostics()["bytes"] <= 8 << 20


def test_budget_exhausted_by_capacity_growth(Extractor):
    """The torus workload needs its vertex arrays grown several times; a 24 MiB
    budget admits the first buffers but not the growth."""
    from paper_2306_07212_gb300.binding import PcError
    net, box = wl.torus_d3()
    with Extractor(precision="mixed", mem_budget_bytes=24 << 20) as ex:
        with pytest.raises(PcError) as e:
            ex.extract(net, box)
        assert e.value.status == 2, str(e.value)
        small, sbox = wl.small_d2()
        ex.extract(small, sbox)
        _same_as_oracle(ex, small, sbox, "after a failed growth")


def test_grid_barrier_wait_runs_out(Extractor):
    from paper_2306_07212_gb300.binding import PcError
    net, box = wl.small_d2()
    with Extractor(precision="mixed", debug_barrier_timeout=True) as ex:
        for _ in range(2):
            with pytest.raises(PcError) as e:
                ex.extract(net, box)
            assert e.value.status == 7, str(e.value)
    # the switch only touches the persistent kernel's barriers: stepwise
    # execution has none and succeeds
    with Extractor(precision="mixed", execution="stepwise", debug_barrier_timeout=True) as ex:
        ex.extract(net, box)
        _same_as_oracle(ex, net, box, "stepwise with the barrier test switch")
    # and an ordinary context on the same device is unaffected
    with Extractor(precision="mixed") as ex:
        ex.extract(net, box)
        _same_as_oracle(ex, net, box, "after barrier timeouts")
