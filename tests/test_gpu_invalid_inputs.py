"""Inputs the library rejects before any device work, and the context staying
usable after each: networks and boxes outside the limits of include/pc.h
(1 <= D <= 8, 1 <= L <= 16, widths <= 256, 2D + neurons <= 1024, hi > lo),
reading results after a failed call, pc_backward without the tape.  Each
rejection is PC_ERR_INVALID (or PC_ERR_NO_TAPE) with a message."""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    with Extractor(precision="mixed") as e:
        yield e


def _net(widths):
    return wl.he_normal_mlp(widths, seed=0)


BAD = [
    ("input dimension 9", _net([9, 4, 1]), wl.Box.cube(9), "input dimension"),
    ("17 layers", _net([2] + [2] * 16 + [1]), wl.Box.cube(2), "number of layers"),
    ("width 257", _net([2, 257, 1]), wl.Box.cube(2), "layer widths"),
    ("1025 entries", _net([2, 256, 256, 256, 256, 1]), wl.Box.cube(2), "<= 1024"),
    ("empty box", _net([2, 4, 1]), wl.Box(np.array([-1.0, 0.5]), np.array([1.0, 0.5])), "hi > lo"),
]


@pytest.mark.parametrize("what,net,box,msg", BAD, ids=[b[0] for b in BAD])
def test_rejected_before_device_work(ex, what, net, box, msg):
    from paper_2306_07212_gb300.binding import PcError
    with pytest.raises(PcError) as e:
        ex.extract(net, box)
    assert e.value.status == 1 and msg in str(e.value), str(e.value)
    with pytest.raises(PcError) as e:  # a failed call leaves no result to read
        ex.counts()
    assert e.value.status == 1 and "no extraction result" in str(e.value)


def test_backward_without_tape(ex):
    from paper_2306_07212_gb300.binding import PcError
    net, box = wl.small_d2()
    ex.extract(net, box)
    c = ex.counts()
    gx = np.zeros((c["D"], c["nV"]))
    gp = np.zeros(net.flat_params().size)
    with pytest.raises(PcError) as e:
        ex.backward(gx, gp)
    assert e.value.status == 8


def test_context_usable_after_rejections(ex):
    net, box = wl.small_d2()
    ref = oracle.extract(net, box)
    ex.extract(net, box)
    c = ex.counts()
    got = (ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges())
    assert_same_complex(got, (ref.X, ref.S, ref.E), coord_tol=1e-6 * 2 * np.sqrt(2), what="after rejections")
