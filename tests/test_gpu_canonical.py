"""Canonical output order (pc_options.canonical): the sorted result is the
oracle's complex, is in the documented order, and is identical from run to
run (without it, edge order and vertex numbering depend on the scheduling of
the pairing step)."""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


def _result(ex):
    c = ex.counts()
    return ex.vertices(), ex.sign_words(), ex.edges(), ex.values(), c["P"]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("widths", [[2, 8, 8, 1], [3, 16, 16, 16, 1], [4, 12, 12, 1]])
def test_canonical_order(cuda, precision, widths):
    net = wl.he_normal_mlp(widths, seed=21)
    box = wl.Box.cube(widths[0])
    ref = oracle.extract(net, box)
    runs = []
    for _ in range(2):
        with cuda(precision=precision, canonical=True) as ex:
            ex.extract(net, box)
            runs.append(_result(ex))
    (X, W, E, Z, P), (X2, W2, E2, Z2, _) = runs
    # identical arrays from run to run
    assert np.array_equal(W, W2) and np.array_equal(E, E2)
    assert np.array_equal(X, X2) and np.array_equal(Z, Z2)
    # vertices sorted by sign words (word 0 most significant, unsigned)
    keys = [tuple(int(x) for x in col) for col in W.T]
    assert all(a < b for a, b in zip(keys, keys[1:])), "vertices not in strictly increasing sign-word order"
    # edges as (smaller, larger), sorted
    assert np.all(E[:, 0] < E[:, 1])
    ek = E[:, 0].astype(np.int64) * (1 << 32) + E[:, 1]
    assert np.all(np.diff(ek) > 0)
    # the oracle's complex
    tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    assert_same_complex((X, unpack_codes(W, P), E), (ref.X, ref.S, ref.E), coord_tol=tol, what=f"{widths} canonical")
    # values follow their vertices: compare with an unsorted run by sign vector
    with cuda(precision=precision) as ex:
        ex.extract(net, box)
        X0, W0, E0, Z0, _ = _result(ex)
    pos = {col.tobytes(): i for i, col in enumerate(np.ascontiguousarray(W0.T))}
    idx = np.array([pos[col.tobytes()] for col in np.ascontiguousarray(W.T)])
    assert np.array_equal(Z, Z0[idx])
    assert np.array_equal(X, X0[idx])


def test_canonical_rejects_keep_tape(cuda):
    from paper_2306_07212_gb300.binding import PcError
    with pytest.raises(PcError):
        cuda(canonical=True, keep_tape=True)
