"""GPU face poset (pc_build_poset / pc_poset_level, Section 4.1) against the
oracle's, element by element.

For every level k the cells' sign vectors must be the oracle's (as sets),
and for every k-cell its parents -- the (k+1)-cells obtained by perturbing
its zeros in entry order, + before -, a box facet's zero only toward + --
must be the oracle's parents of the same cell, in the same order, after
both sides' cells are matched by sign vector.  On the D=3 torus workload,
where the oracle's poset is slow, the counts must equal pc_cell_counts and
every cell's number of parents the count of Section 4.1, z + 2 (D - k - z)
for z zeros at box facets.
"""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import unpack_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Extractor():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


def _index(cells):
    return {tuple(c): i for i, c in enumerate(map(tuple, cells))}


def _compare(gpu, orc, P, D, what):
    cg = [unpack_codes(c.T, P) for c, _, _ in gpu]
    for k in range(D + 1):
        assert cg[k].shape == orc.cells[k].shape, f"{what}: level {k} has {len(cg[k])} cells, oracle {len(orc.cells[k])}"
        oi = _index(orc.cells[k])
        assert len(oi) == len(cg[k])
        perm = np.array([oi.get(tuple(c), -1) for c in cg[k]])
        assert np.all(perm >= 0), f"{what}: level {k} has cells the oracle does not"
        assert len(set(perm.tolist())) == len(perm)
        if k == D:
            break
        rp, cols = gpu[k][1], gpu[k][2]
        orp, ocl = orc.parents[k]
        up = np.array([_index(orc.cells[k + 1]).get(tuple(c), -1) for c in cg[k + 1]])
        for i in range(len(cg[k])):
            mine = up[cols[rp[i]:rp[i + 1]]]
            j = perm[i]
            theirs = ocl[orp[j]:orp[j + 1]]
            assert np.array_equal(mine, theirs), f"{what}: parents of {k}-cell {i} differ"


CASES = [("small_d2", *wl.small_d2())] + [
    (f"D{D}-{w}x{d}", wl.he_normal_mlp([D] + [w] * d + [1], seed=70 + s), wl.Box.cube(D))
    for s, (D, w, d) in enumerate([(2, 12, 2), (3, 8, 2), (3, 6, 3), (4, 6, 2)])]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,net,box", CASES, ids=[c[0] for c in CASES])
def test_poset_matches_oracle(Extractor, precision, name, net, box):
    ref = oracle.extract(net, box)
    assert ref.status == 0, ref.error
    orc = oracle.poset(ref)
    assert orc.status == 0, orc.error
    with Extractor(precision=precision) as ex:
        ex.extract(net, box)
        P = ex.counts()["P"]
        gpu = ex.poset()
        # levels 0 and 1 follow the vertex and edge order of the result
        S_words = ex.sign_words()
        assert np.array_equal(gpu[0][0], S_words.T)
        E = ex.edges()
        assert np.array_equal(gpu[1][0], S_words.T[E[:, 0]] | S_words.T[E[:, 1]])
    _compare(gpu, orc, P, net.D, f"{name} {precision}")


def test_poset_on_the_torus(Extractor):
    net, box = wl.torus_d3()
    with Extractor(precision="mixed") as ex:
        ex.extract(net, box)
        f, chi = ex.cell_counts()
        P = ex.counts()["P"]
        gpu = ex.poset()
    D = net.D
    assert [len(c) for c, _, _ in gpu] == list(f) and chi == 1
    for k in range(D):
        cells = unpack_codes(gpu[k][0].T, P)
        zeros = cells == 0
        zb = zeros[:, :2 * D].sum(axis=1)
        z = zeros.sum(axis=1)
        assert np.all(z == D - k)
        expect = zb + 2 * (z - zb)  # facet zeros: one parent each; neuron zeros: two
        assert np.array_equal(np.diff(gpu[k][1]), expect), f"level {k}: parent counts"
        assert gpu[k][2].min() >= 0 and gpu[k][2].max() < len(gpu[k + 1][0])


def test_poset_is_invalid_after_the_next_extraction(Extractor):
    from paper_2306_07212_gb300.binding import PcError
    net, box = wl.small_d2()
    with Extractor(precision="fp64") as ex:
        ex.extract(net, box)
        ex.poset()
        ex.extract(net, box)
        with pytest.raises(PcError):
            n = __import__("ctypes").c_int64()
            ex._check(ex._lib.pc_poset_level(ex._ctx, 0, __import__("ctypes").byref(n), None, None, None, None))
