"""Region counts of generic hyperplane arrangements clipped to a convex
domain, against the oracle's k-face counts by perturbation (Section 4.1).

For n hyperplanes in general position and a convex domain K, every region
of the clipped arrangement is counted once by the lowest point of its
closure in a generic direction, which gives
    regions = sum over k = 0..D of #{k-subsets whose flats meet the open K}
(the empty subset counts once).  A single-layer network [D, n] is such an
arrangement; the subset flats are checked with plain linear algebra and a
small linear program per flat (scipy), independent of the oracle.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl

linprog = pytest.importorskip("scipy.optimize").linprog


def _flat_meets_open_domain(W, b, A, c):
    """Does {x : W x + b = 0} meet {x : c - A x > 0}?  Maximise the slack s
    of c - A x >= s on the flat (s <= 1); the open domain is met iff s > 0."""
    D = A.shape[1]
    obj = np.zeros(D + 1)
    obj[-1] = -1.0
    A_ub = np.hstack([A, np.ones((A.shape[0], 1))])
    A_eq = np.hstack([W, np.zeros((W.shape[0], 1))]) if len(W) else None
    res = linprog(obj, A_ub=A_ub, b_ub=c, A_eq=A_eq, b_eq=(-b if len(W) else None),
                  bounds=[(None, None)] * D + [(None, 1.0)], method="highs")
    return res.status == 0 and -res.fun > 1e-9


def _regions(W, b, A, c):
    D = A.shape[1]
    total = 1
    for k in range(1, D + 1):
        for sub in itertools.combinations(range(len(W)), k):
            if _flat_meets_open_domain(W[list(sub)], b[list(sub)], A, c):
                total += 1
    return total


@pytest.mark.parametrize("D,n", [(2, 6), (2, 15), (3, 5), (3, 9), (4, 6), (5, 6)])
@pytest.mark.parametrize("domain", ["box", "simplex", "corner_cut"])
def test_regions_of_a_clipped_arrangement(D, n, domain):
    net = wl.he_normal_mlp([D, n], seed=10 * D + n, bias_var=0.25)
    if domain == "box":
        box = wl.Box.cube(D)
        dom = wl.Polytope.from_box(box)
        r = oracle.extract(net, box)
    else:
        dom = getattr(wl.Polytope, domain)(D)
        r = oracle.extract_domain(net, dom)
    assert r.status == 0
    f, chi = oracle.faces(r)
    assert chi == 1
    assert f[D] == _regions(net.W[0], net.b[0], dom.A, dom.c)
