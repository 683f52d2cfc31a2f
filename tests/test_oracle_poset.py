"""Pins of the oracle's face poset (Section 4.1: the cells of the complex by
perturbation, each cell's parents by perturbing one of its zeros), against
what the mathematics of polyhedral complexes fixes, independently of how the
poset is built:

* the vertices' perturbations are exactly the edges of the extraction (built
  separately, as the joins of the edges' endpoints);
* every k-cell has D - k zeros and lies on the cells above it (one zero
  becomes nonzero, nothing else changes);
* diamond property: between a (k-2)-cell and a k-cell that contains it
  there are exactly two (k-1)-cells;
* the boundary of every k-cell is a (k-1)-sphere: the alternating sum of its
  faces' counts is 1 - (-1)^k;
* geometry: the centroid of a cell's vertices, evaluated by a plain numpy
  forward pass, has the cell's sign vector (nonzero entries), and its zero
  entries vanish there (convex cells contain their vertex centroid in their
  relative interior);
* the level counts equal the perturbation counts of orc_faces (Euler
  characteristic 1).
"""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import entry_values


def _children(q, k):
    """CSR of the (k-1)-cells below each k-cell (inverse of parents[k-1])."""
    rp, cl = q.parents[k - 1]
    n_child = len(q.cells[k - 1])
    rows = np.repeat(np.arange(n_child), np.diff(rp))
    order = np.argsort(cl, kind="stable")
    ch_rp = np.zeros(len(q.cells[k]) + 1, np.int64)
    np.add.at(ch_rp, cl + 1, 1)
    return np.cumsum(ch_rp), rows[order]


def _check_poset(net, box, res, D, check_geometry=True, q=None):
    q = q if q is not None else oracle.poset(res)
    assert q.status == 0, q.error
    f, chi = oracle.faces(res)
    assert [len(c) for c in q.cells] == list(f) and chi == 1
    assert len(q.cells[0]) == res.nV
    for k, c in enumerate(q.cells):
        assert np.all(np.sum(c == 0, axis=1) == D - k), f"level {k}: wrong number of zeros"
    # the vertices' parents are the extraction's edges (joins built separately)
    V = res.S
    order = np.lexsort(V.T[::-1])
    rank = np.empty(len(order), np.int64)
    rank[order] = np.arange(len(order))
    assert np.array_equal(q.cells[0], V[order])
    rp, cl = q.parents[0]
    pairs = set()
    for v in range(len(q.cells[0])):
        for e in cl[rp[v]:rp[v + 1]]:
            pairs.add((v, int(e)))
    E = rank[res.E]
    joins = np.where(res.S[res.E[:, 0]] != 0, res.S[res.E[:, 0]], res.S[res.E[:, 1]])
    eidx = {tuple(s): i for i, s in enumerate(map(tuple, q.cells[1]))}
    expect = set()
    for (a, b), s in zip(E, joins):
        j = eidx[tuple(s)]
        expect.add((int(a), j))
        expect.add((int(b), j))
    assert pairs == expect, "vertex perturbations differ from the extraction's edges"
    # parents: one zero becomes nonzero, nothing else changes
    for k in range(D):
        rp, cl = q.parents[k]
        rows = np.repeat(np.arange(len(q.cells[k])), np.diff(rp))
        lo, hi = q.cells[k][rows].astype(np.int16), q.cells[k + 1][cl].astype(np.int16)
        diff = lo != hi
        assert np.all(diff.sum(axis=1) == 1) and np.all(lo[diff] == 0)
    # diamonds: every (k-2, k) interval has exactly two cells in between
    for k in range(2, D + 1):
        rp0, cl0 = q.parents[k - 2]
        rp1, cl1 = q.parents[k - 1]
        for a in range(len(q.cells[k - 2])):
            mids = cl0[rp0[a]:rp0[a + 1]]
            tops = np.concatenate([cl1[rp1[g]:rp1[g + 1]] for g in mids]) if len(mids) else np.zeros(0, np.int64)
            _, counts = np.unique(tops, return_counts=True)
            assert np.all(counts == 2), f"level {k - 2} cell {a}: an interval is not a diamond"
    # boundary spheres: faces of each k-cell, alternating sum 1 - (-1)^k
    ch = {k: _children(q, k) for k in range(1, D + 1)}
    for k in range(1, D + 1):
        for c in range(len(q.cells[k])):
            below = {k: {c}}
            for j in range(k, 0, -1):
                crp, ccl = ch[j]
                below[j - 1] = {int(x) for y in below[j] for x in ccl[crp[y]:crp[y + 1]]}
            s = sum((-1) ** j * len(below[j]) for j in range(k))
            assert s == 1 - (-1) ** k, f"{k}-cell {c}: boundary Euler characteristic {s}"
            if check_geometry:
                verts = np.array(sorted(below[0]))
                x = res.X[order[verts]].mean(axis=0)
                vals = entry_values(net, box, x[None, :])[0]
                sig = q.cells[k][c]
                nz = sig != 0
                scale = 1.0 + np.abs(vals).max()
                assert np.all(np.sign(vals[nz]) == sig[nz]), f"{k}-cell {c}: centroid outside the cell"
                assert np.all(np.abs(vals[~nz]) <= 1e-9 * scale), f"{k}-cell {c}: centroid off its zero set"
    return q


NETS = [("small_d2", *wl.small_d2())] + [
    (f"D{D}-{w}x{d}-s{s}", wl.he_normal_mlp([D] + [w] * d + [1], seed=s), wl.Box.cube(D))
    for s, (D, w, d) in enumerate([(2, 6, 2), (2, 10, 1), (3, 5, 2), (3, 4, 3), (4, 4, 1), (4, 3, 2), (3, 8, 1)])]


@pytest.mark.parametrize("name,net,box", NETS, ids=[n[0] for n in NETS])
def test_poset_pins(name, net, box):
    res = oracle.extract(net, box)
    assert res.status == 0, res.error
    _check_poset(net, box, res, net.D)


def test_poset_on_a_simplex_domain():
    """A polyhedral domain (Section 4.1): the simplex's facets are perturbed
    only toward the inside, like the box's."""
    net = wl.he_normal_mlp([3, 5, 4, 1], seed=42)
    dom = wl.Polytope.simplex(3)
    res = oracle.extract_domain(net, dom)
    assert res.status == 0, res.error
    q = oracle.poset(res)
    assert q.status == 0, q.error
    f, chi = oracle.faces(res)
    assert [len(c) for c in q.cells] == list(f) and chi == 1


def _corrupt(q, what):
    import copy
    q = copy.deepcopy(q)
    if what == "drop_incidence":  # an edge loses one of its two faces
        rp, cl = q.parents[1]
        cl = cl.copy()
        cl[0] = cl[1] if len(cl) > 1 and cl[1] != cl[0] else cl[0]
        q.parents[1] = (rp, cl)
    elif what == "outward_facet":  # a region's facet entry perturbed outward
        c = q.cells[2].copy()
        j = int(np.nonzero(c[0, :4] == 1)[0][0])
        c[0, j] = -1
        q.cells[2] = c
    return q


@pytest.mark.parametrize("what", ["drop_incidence", "outward_facet"])
def test_poset_pins_fail_on_a_planted_mistake(what):
    """A plausible mistake in a poset (a lost incidence, a box facet's zero
    perturbed outward) fails the pins."""
    net, box = wl.he_normal_mlp([2, 6, 1], seed=3), wl.Box.cube(2)
    res = oracle.extract(net, box)
    q = _corrupt(oracle.poset(res), what)
    with pytest.raises(AssertionError):
        _check_poset(net, box, res, net.D, q=q)
