"""Pins for the oracle on the counting-sweep nets (Section 5.1.2).

The sweep nets (four hidden layers of width 10, 20 or 40, a scalar output,
uniform initialisation, box [-1,1]^D) are checked against constructions that
share nothing with edge subdivision:

* D = 1: every neuron's zeros found layer by layer from the breakpoints of
  the earlier layers (each pre-activation is affine between consecutive
  breakpoints), then the complex is the sorted point set with consecutive
  edges;
* first layer in D = 2..4: the vertex census of a hyperplane arrangement
  clipped by the box, one vertex per (j planes, j-face of the box) whose
  intersection lies in the relative interior of the face, compared as the
  set of zero patterns;
* the stored counts of the golden file are reproduced by the oracle.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import forward_all

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "counting_sweep_counts.json")


def test_sweep_nets_are_drawn_as_stated():
    net, box = wl.counting_sweep_net(3, 20, seed=4)
    assert net.widths == [3, 20, 20, 20, 20, 1]
    assert np.array_equal(box.lo, -np.ones(3)) and np.array_equal(box.hi, np.ones(3))
    for W, b in zip(net.W, net.b):
        bound = 1.0 / np.sqrt(W.shape[1])
        assert np.all(np.abs(W) <= bound) and np.all(np.abs(b) <= bound)
        assert np.array_equal(W.astype(np.float32).astype(np.float64), W)
        # a uniform draw fills its interval: the extremes come near the bound
        assert np.abs(W).max() > 0.8 * bound
    again, _ = wl.counting_sweep_net(3, 20, seed=4)
    other, _ = wl.counting_sweep_net(3, 20, seed=3)
    assert np.array_equal(again.flat_params(), net.flat_params())
    assert not np.array_equal(other.flat_params(), net.flat_params())


# --- D = 1: breakpoint propagation -------------------------------------------

def _breakpoint_scan(net, lo, hi):
    """(x, neuron) for every zero of every neuron on the open interval (lo, hi)."""
    bps = np.array([lo, hi], np.float64)
    out, n0 = [], 0
    for l in range(net.L):
        H = net.widths[l + 1]
        Z = forward_all(net, bps[:, None])[:, n0:n0 + H]
        assert np.all(Z != 0.0), "a zero on a breakpoint (non-generic net)"
        new = []
        for i in range(H):
            z = Z[:, i]
            for k in range(len(bps) - 1):
                a, b = z[k], z[k + 1]
                if (a > 0) != (b > 0):
                    new.append((bps[k] + (bps[k + 1] - bps[k]) * a / (a - b), n0 + i))
        out.extend(new)
        bps = np.sort(np.concatenate([bps, [x for x, _ in new]]))
        n0 += H
    return out


@pytest.mark.parametrize("width", wl.COUNTING_WIDTHS)
@pytest.mark.parametrize("seed", range(wl.COUNTING_SEEDS))
def test_d1_complex_is_the_breakpoint_scan(width, seed):
    net, box = wl.counting_sweep_net(1, width, seed)
    r = oracle.extract(net, box)
    assert r.status == 0, r.error
    scan = sorted(_breakpoint_scan(net, -1.0, 1.0))
    xs = np.array([-1.0] + [x for x, _ in scan] + [1.0])
    order = np.argsort(r.X[:, 0], kind="stable")
    assert r.nV == len(xs)
    assert np.max(np.abs(r.X[order, 0] - xs)) < 1e-10
    # the zero entry of each interior vertex is the neuron the scan found
    S = r.S[order]
    assert S[0, 0] == 0 and S[-1, 1] == 0
    for k, (_, n) in enumerate(scan, start=1):
        assert S[k, 2 + n] == 0, f"vertex {k} does not lie on neuron {n}"
        assert np.count_nonzero(S[k] == 0) == 1
    # edges join neighbours on the line, each pair once
    rank = np.empty(r.nV, np.int64)
    rank[order] = np.arange(r.nV)
    Er = np.sort(rank[r.E.astype(np.int64)], axis=1)
    Er = Er[np.lexsort((Er[:, 1], Er[:, 0]))]
    assert np.array_equal(Er, np.stack([np.arange(r.nV - 1), np.arange(1, r.nV)], axis=1))


# --- first layer: clipped arrangement census ---------------------------------

def _clipped_arrangement_zero_patterns(W, b, D):
    """Zero patterns (facet entries, plane indices) of every vertex of the
    arrangement {W x + b = 0} inside [-1,1]^D."""
    H = W.shape[0]
    pats = set()
    for j in range(D + 1):
        for fixed in itertools.combinations(range(D), D - j):
            free = [d for d in range(D) if d not in fixed]
            for sides in itertools.product((0, 1), repeat=D - j):
                xf = np.array([(-1.0, 1.0)[s] for s in sides])
                facets = tuple(sorted(2 * d + s for d, s in zip(fixed, sides)))
                if j == 0:
                    pats.add((facets, ()))
                    continue
                for T in itertools.combinations(range(H), j):
                    A = W[list(T)][:, free]
                    rhs = -(b[list(T)] + W[list(T)][:, list(fixed)] @ xf)
                    try:
                        y = np.linalg.solve(A, rhs)
                    except np.linalg.LinAlgError:
                        continue
                    if np.all(np.abs(y) < 1.0):
                        pats.add((facets, T))
    return pats


@pytest.mark.parametrize("D,width", [(2, 10), (2, 40), (3, 10), (3, 20), (4, 10)])
def test_first_layer_vertices_are_the_clipped_arrangement(D, width):
    net, box = wl.counting_sweep_net(D, width, seed=0)
    r = oracle.extract(net, box, max_neurons=width)
    assert r.status == 0, r.error
    m = 2 * D
    got = set()
    for s in r.S:
        z = np.nonzero(s[:m + width] == 0)[0]
        got.add((tuple(int(k) for k in z[z < m]), tuple(int(k) - m for k in z[z >= m])))
    assert len(got) == r.nV, "two vertices share a zero pattern"
    want = _clipped_arrangement_zero_patterns(net.W[0], net.b[0], D)
    assert got == want


# --- golden counts ---------------------------------------------------------------

def test_golden_counts_are_the_oracles():
    with open(GOLDEN) as f:
        doc = json.load(f)
    checked = 0
    for p in doc["points"]:
        if p["D"] > 3 or (p["D"] == 3 and p["width"] == 40):
            continue  # larger points take the oracle seconds each
        for row in p["counts"][:2]:
            net, box = wl.counting_sweep_net(p["D"], p["width"], row["seed"])
            r = oracle.extract(net, box)
            assert (r.nV, r.nE) == (row["nV"], row["nE"]), (p["D"], p["width"], row["seed"])
            checked += 1
    assert checked >= 12
