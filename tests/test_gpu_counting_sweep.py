"""The counting sweep of Section 5.1.2 on the GPU: randomly initialised nets of
four hidden layers (widths 10, 20, 40) and a scalar output on [-1,1]^D.

Where the oracle finishes in about a second the complexes must be identical
(sign vectors and edges bit-exact, coordinates within 1e-6 of the box
diameter).  At every point of the stored oracle counts up to D = 4 (five nets
per point, the largest about 1.3e6 vertices and 5e6 edges) the vertex and
edge counts must equal the oracle's, and properties that hold at any size are
checked on the largest point.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, entry_values, unpack_codes

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "counting_sweep_counts.json")
GPU_DIMS = (1, 2, 3, 4)


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


def _triple(ex):
    c = ex.counts()
    return ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges()


@pytest.mark.parametrize("D,width", [(1, 10), (1, 20), (1, 40), (2, 10), (2, 20), (2, 40), (3, 10), (3, 20),
                                     (3, 40), (4, 10), (4, 20)])
def test_sweep_point_matches_oracle(cuda, D, width):
    for seed in range(2):
        net, box = wl.counting_sweep_net(D, width, seed)
        ref = oracle.extract(net, box)
        assert ref.status == 0, ref.error
        tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
        with cuda(precision="mixed") as ex:
            ex.extract(net, box)
            assert_same_complex(_triple(ex), (ref.X, ref.S, ref.E), coord_tol=tol,
                                what=f"D={D} width={width} seed={seed}")


def test_sweep_counts_match_stored_oracle_counts(cuda):
    with open(GOLDEN) as f:
        doc = json.load(f)
    checked = 0
    with cuda(precision="mixed") as ex:
        for p in doc["points"]:
            if p["D"] not in GPU_DIMS:
                continue
            for row in p["counts"]:
                net, box = wl.counting_sweep_net(p["D"], p["width"], row["seed"])
                ex.extract(net, box)
                c = ex.counts()
                assert (c["nV"], c["nE"]) == (row["nV"], row["nE"]), (p["D"], p["width"], row["seed"])
                checked += 1
    assert checked >= 12 * wl.COUNTING_SEEDS


def test_largest_sweep_point_properties(cuda):
    net, box = wl.counting_sweep_net(4, 40, 0)
    with cuda(precision="mixed") as ex:
        ex.extract(net, box)
        X, S, E = _triple(ex)
    D, m = 4, 8
    assert np.all((S == 0).sum(axis=1) == D)
    deg = np.bincount(E.ravel(), minlength=len(X))
    assert np.array_equal(deg, 2 * D - (S[:, :m] == 0).sum(axis=1))
    # a vertex within the coordinate tolerance (1e-6 of the diameter in every
    # coordinate) of its exact position leaves at most Lip * |dx|_2 on its zero
    # entries; Lip bounds every pre-activation's gradient (ReLU masks contract)
    norms = [np.linalg.norm(W, 2) for W in net.W]
    lip = max([1.0] + [float(np.prod(norms[:k])) for k in range(1, net.L + 1)])
    bound = lip * np.sqrt(D) * 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    rows = np.arange(0, len(X), max(1, len(X) // 20000))
    vals = entry_values(net, box, X[rows])
    assert np.max(np.abs(vals[S[rows] == 0])) < bound
