"""The counting sweep of Section 5.1.2 at D = 5 and up on the GPU (libpc.so
takes D <= 8, its PC_MAX_D=10 build D <= 10): identical complexes for one
width-10 net per D = 5..9, and vertex and edge counts equal to the stored
oracle counts at every stored point with D >= 5 (five nets each; the
largest hold about 1e7 to 3e7 vertices and 5e7 to 1.3e8 edges)."""
import functools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "counting_sweep_counts.json")


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


@functools.lru_cache(maxsize=None)
def _oracle(D):
    net, box = wl.counting_sweep_net(D, 10, seed=0)
    return net, box, oracle.extract(net, box)


def _triple(ex):
    c = ex.counts()
    return ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("D", [5, 6, 7, 8, 9])
def test_high_dim_point_matches_oracle(cuda, D, precision):
    net, box, ref = _oracle(D)
    assert ref.status == 0, ref.error
    with cuda(precision=precision, max_dim=8 if D <= 8 else 10) as ex:
        ex.extract(net, box)
        X, S, E = _triple(ex)
    assert_same_complex((X, S, E), (ref.X, ref.S, ref.E), coord_tol=1e-6 * 2 * np.sqrt(D),
                        what=f"D={D} width=10 {precision}")
    m = 2 * D
    assert np.array_equal(np.bincount(E.ravel(), minlength=len(X)), 2 * D - (S[:, :m] == 0).sum(axis=1))


def test_high_dim_counts_match_stored_oracle_counts(cuda):
    with open(GOLDEN) as f:
        doc = json.load(f)
    checked = 0
    with cuda(precision="mixed") as ex8, cuda(precision="mixed", max_dim=10) as ex10:
        for p in doc["points"]:
            if p["D"] < 5:
                continue
            ex = ex8 if p["D"] <= 8 else ex10
            for row in p["counts"]:
                net, box = wl.counting_sweep_net(p["D"], p["width"], row["seed"])
                ex.extract(net, box)
                c = ex.counts()
                assert (c["nV"], c["nE"]) == (row["nV"], row["nE"]), (p["D"], p["width"], row["seed"])
                checked += 1
    assert checked >= 4 * wl.COUNTING_SEEDS
