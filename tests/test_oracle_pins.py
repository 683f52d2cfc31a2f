"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each check is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a missing pairing) fails
at least one of them:

* brute force from the definition (every D-subset of entries under every
  activation pattern, edges by a midpoint test) on tiny deep nets;
* the closed form of a clipped line arrangement in D=2 and the C(n, D)
  interior-vertex count of a generic arrangement;
* invariants of Section 4.1 (zero counts, vertex degree z + 2(D - k - z)),
  the bookkeeping of steps (4)-(5), the Euler characteristic 1 of the box;
* the zero-residual validation of Section 5.1.1 and a direct D x D solve;
* metamorphic invariance under neuron permutation and positive rescaling;
* the paper's printed 2D counts (Section 5.4.2) against the line-arrangement
  identity, which pins the convention that boundary cells are counted.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, entry_values, solve_vertex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _triple(r):
    return (r.X, r.S, r.E)


# --- brute force ------------------------------------------------------------

TINY = [
    (1, [1, 4, 3, 1]),
    (1, [1, 6, 1]),
    (2, [2, 4, 3, 1]),
    (2, [2, 5, 4, 1]),
    (2, [2, 3, 3, 3, 1]),
    (3, [3, 4, 3, 1]),
    (3, [3, 5, 3, 2]),
    (3, [3, 3, 3, 3, 1]),
]


@pytest.mark.parametrize("D,widths", TINY)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_brute_force_tiny_deep(D, widths, seed):
    net = wl.he_normal_mlp(widths, seed=100 * seed + len(widths))
    box = wl.Box.cube(D)
    r = oracle.extract(net, box)
    assert r.status == 0, r.error
    b = oracle.brute(net, box, tol=1e-9)
    assert b.status == 0, b.error
    assert_same_complex(_triple(r), _triple(b), coord_tol=1e-9, what=f"{widths} seed {seed}")


HIGH = [(4, [4, 3, 2, 1]), (5, [5, 3, 1]), (5, [5, 2, 2, 1]), (6, [6, 3, 1]), (6, [6, 2, 2, 1]),
        (7, [7, 2, 1]), (8, [8, 2, 1]), (8, [8, 2, 1, 1])]


@pytest.mark.parametrize("D,widths", HIGH)
@pytest.mark.parametrize("seed", [0, 1])
def test_matches_brute_force_up_to_d8(D, widths, seed):
    # the dimensions of the counting sweep that the library takes (D <= 8)
    net = wl.he_normal_mlp(widths, seed=50 + seed)
    box = wl.Box.cube(D)
    r = oracle.extract(net, box)
    b = oracle.brute(net, box, tol=1e-9)
    assert r.status == 0 and b.status == 0, (r.error, b.error)
    assert_same_complex(_triple(r), _triple(b), coord_tol=1e-9, what=f"{widths} seed {seed}")


@pytest.mark.slow
def test_small_d2_config_matches_brute_force():
    net, box = wl.small_d2()
    r = oracle.extract(net, box)
    b = oracle.brute(net, box, tol=1e-9)
    assert r.status == 0 and b.status == 0
    assert_same_complex(_triple(r), _triple(b), coord_tol=1e-9, what="2-8-8-1")


# --- closed forms -------------------------------------------------------------

def _line_arrangement_counts(W, b, lo, hi):
    """n_in: lines meeting the open box; I: pairwise intersections inside."""
    n = W.shape[0]
    corners = np.array([[lo[0], lo[1]], [lo[0], hi[1]], [hi[0], lo[1]], [hi[0], hi[1]]])
    vals = corners @ W.T + b
    meets = (vals.max(axis=0) > 0) & (vals.min(axis=0) < 0)
    I = 0
    for i in range(n):
        for j in range(i + 1, n):
            x = np.linalg.solve(np.stack([W[i], W[j]]), -np.array([b[i], b[j]]))
            if np.all(x > lo) and np.all(x < hi):
                I += 1
    return int(meets.sum()), I


@pytest.mark.parametrize("n", [1, 3, 7, 16, 30])
@pytest.mark.parametrize("seed", [0, 1])
def test_line_arrangement_closed_form(n, seed):
    net = wl.he_normal_mlp([2, n], seed=seed, bias_var=0.25)
    box = wl.Box.cube(2)
    r = oracle.extract(net, box)
    assert r.status == 0
    n_in, I = _line_arrangement_counts(net.W[0], net.b[0], box.lo, box.hi)
    assert r.nV == 4 + 2 * n_in + I
    assert r.nE == 4 + 3 * n_in + 2 * I


@pytest.mark.parametrize("D,n", [(2, 9), (3, 7), (4, 6)])
def test_generic_arrangement_interior_vertices(D, n):
    net = wl.he_normal_mlp([D, n], seed=7)
    W, b = net.W[0], net.b[0]
    pts = []
    import itertools
    for sub in itertools.combinations(range(n), D):
        pts.append(np.linalg.solve(W[list(sub)], -b[list(sub)]))
    half = 1.5 * np.max(np.abs(pts)) + 1.0
    r = oracle.extract(net, wl.Box.cube(D, half))
    assert r.status == 0
    interior = np.all(r.S[:, :2 * D] == 1, axis=1)
    assert interior.sum() == math.comb(n, D)


def test_paper_printed_2d_counts_fit_line_arrangement():
    """Section 5.4.2 prints per-layer counts for a trained 2-50-50-1 net.

    The first layer is a line arrangement, so V = 4 + 2 n_in + I and
    E = 4 + 3 n_in + 2 I must have a solution in integers with
    0 <= n_in <= 50 and 0 <= I <= C(n_in, 2) when box vertices and edges are
    counted.  The last (one-neuron) step adds a closed level curve, for which
    every new vertex also brings one intersecting edge: dE = 2 dV.
    """
    with open(os.path.join(GOLDEN, "paper_2d_counts.json")) as f:
        g = json.load(f)
    V1, E1 = g["vertices_per_layer"][0], g["edges_per_layer"][0]
    n_in = 2 * V1 - E1 - 4
    I = V1 - 4 - 2 * n_in
    assert 0 <= n_in <= 50 and 0 <= I <= math.comb(n_in, 2)
    dV = g["vertices_per_layer"][2] - g["vertices_per_layer"][1]
    dE = g["edges_per_layer"][2] - g["edges_per_layer"][1]
    assert dE == 2 * dV


# --- invariants ------------------------------------------------------------

INV = [(2, [2, 12, 12, 1], 0), (2, [2, 16, 16, 16, 1], 1), (3, [3, 10, 10, 1], 2),
       (3, [3, 16, 16, 1], 3), (4, [4, 8, 8, 1], 4)]


@pytest.mark.parametrize("D,widths,seed", INV)
def test_invariants(D, widths, seed):
    _check_invariants(wl.he_normal_mlp(widths, seed=seed), wl.Box.cube(D))


@pytest.mark.parametrize("D,width,seed", [(2, 20, 0), (2, 40, 1), (3, 10, 2), (3, 20, 3), (4, 10, 4)])
def test_invariants_counting_sweep_nets(D, width, seed):
    # uniformly initialised nets of four hidden layers (Section 5.1.2)
    _check_invariants(*wl.counting_sweep_net(D, width, seed))


def _check_invariants(net, box):
    D = net.D
    r = oracle.extract(net, box)
    assert r.status == 0, r.error
    m = 2 * D
    # I1: every vertex has exactly D zeros; every edge (join) exactly D-1.
    assert np.all((r.S == 0).sum(axis=1) == D)
    Su, Sw = r.S[r.E[:, 0]], r.S[r.E[:, 1]]
    assert not np.any((Su != 0) & (Sw != 0) & (Su != Sw)), "edge endpoints not conformal"
    join = np.where(Su != 0, Su, Sw)
    assert np.all((join == 0).sum(axis=1) == D - 1)
    # I2: a vertex has z + 2(D - z) parent edges, z = its boundary zeros.
    deg = np.bincount(r.E.ravel(), minlength=r.nV)
    zb = (r.S[:, :m] == 0).sum(axis=1)
    assert np.array_equal(deg, 2 * D - zb)
    # I3/I4: per neuron, every 2-face key paired exactly twice.
    nsplit, nkeys, npairs, ndeg = r.stats.T
    assert np.all(nkeys == 2 * npairs) and np.all(ndeg == 0)
    assert r.nV == 2 ** D + nsplit.sum()
    assert r.nE == D * 2 ** (D - 1) + nsplit.sum() + npairs.sum()
    # I5: the subdivided box is a closed ball, Euler characteristic 1.
    f, chi = oracle.faces(r)
    assert chi == 1, f"face counts {f}"
    # I6: zero entries evaluate to ~0 at the vertex (Section 5.1.1); nonzero
    # entries have the recorded sign.
    vals = entry_values(net, box, r.X)
    zero = r.S == 0
    assert np.max(np.abs(vals[zero])) < 1e-12
    assert np.all(np.sign(vals[~zero]) == r.S[~zero])
    # I7: coordinates equal a direct solve of the vertex's zero entries.
    for v in range(0, r.nV, max(1, r.nV // 200)):
        x = solve_vertex(net, box, r.S[v])
        assert np.max(np.abs(x - r.X[v])) < 1e-12


def test_every_layer_processed_including_output():
    net = wl.he_normal_mlp([2, 6, 6, 3], seed=11)
    r = oracle.extract(net, wl.Box.cube(2))
    # neurons of the output layer own sign entries, and some vertex lies on them
    m = 4
    out = r.S[:, m + 12:]
    assert out.shape[1] == 3
    assert np.any(out == 0)


def test_prefix_extraction_is_the_smaller_net():
    """Stopping after the first layer equals extracting the one-layer net."""
    net = wl.he_normal_mlp([3, 8, 8, 1], seed=5)
    box = wl.Box.cube(3)
    r = oracle.extract(net, box, max_neurons=8)
    one = wl.Net([3, 8], [net.W[0]], [net.b[0]])
    s = oracle.extract(one, box)
    assert_same_complex((r.X, r.S[:, :6 + 8], r.E), _triple(s), coord_tol=0, what="prefix")


# --- metamorphic -------------------------------------------------------------

@pytest.mark.parametrize("D,widths", [(2, [2, 10, 10, 1]), (3, [3, 8, 8, 1])])
def test_neuron_permutation_invariance(D, widths):
    net = wl.he_normal_mlp(widths, seed=21)
    box = wl.Box.cube(D)
    r = oracle.extract(net, box)
    rng = np.random.default_rng(3)
    perm = rng.permutation(widths[1])
    W0, b0, W1 = net.W[0][perm], net.b[0][perm], net.W[1][:, perm]
    pnet = wl.Net(list(widths), [W0, W1] + net.W[2:], [b0] + net.b[1:])
    p = oracle.extract(pnet, box)
    m = 2 * D
    cols = np.arange(r.S.shape[1])
    cols[m:m + widths[1]] = m + np.argsort(perm)
    # entry m+k of the permuted net is neuron perm[k] of the original
    Sp_back = p.S.copy()
    Sp_back[:, m:m + widths[1]] = p.S[:, m + np.argsort(perm)]
    assert_same_complex(_triple(r), (p.X, Sp_back, p.E), coord_tol=1e-12, what="permutation")


@pytest.mark.parametrize("D,widths", [(2, [2, 10, 10, 1]), (3, [3, 8, 8, 1])])
def test_positive_rescaling_invariance(D, widths):
    net = wl.he_normal_mlp(widths, seed=22)
    box = wl.Box.cube(D)
    r = oracle.extract(net, box)
    c = np.exp(np.random.default_rng(4).uniform(-2, 2, widths[1]))
    snet = wl.Net(list(widths), [net.W[0] * c[:, None], net.W[1] / c[None, :]] + net.W[2:],
                  [net.b[0] * c] + net.b[1:])
    s = oracle.extract(snet, box)
    assert_same_complex(_triple(r), _triple(s), coord_tol=1e-12, what="rescaling")


# --- gradient ----------------------------------------------------------------

def _sphere_loss(res, D):
    on = res.S[:, -1] == 0
    x = res.X
    rad = np.linalg.norm(x, axis=1)
    L = np.sum(np.where(on, (rad - 1.0) ** 2, 0.0))
    gx = np.where(on[:, None], 2 * (rad - 1.0)[:, None] * x / np.maximum(rad, 1e-300)[:, None], 0.0)
    return L, gx


def test_implicit_gradient_matches_finite_differences():
    net = wl.he_normal_mlp([3, 8, 8, 1], seed=9)
    box = wl.Box.cube(3)
    r = oracle.extract(net, box)
    L0, gx = _sphere_loss(r, 3)
    g = oracle.grad(net, r, gx)
    theta = net.flat_params()
    rng = np.random.default_rng(0)
    idx = rng.choice(theta.size, 24, replace=False)
    h = 1e-6
    checked = 0
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        rp = oracle.extract(net.with_flat_params(tp), box)
        rm = oracle.extract(net.with_flat_params(tm), box)
        if rp.nV != r.nV or rm.nV != r.nV:
            continue  # combinatorics changed: finite difference undefined
        fd = (_sphere_loss(rp, 3)[0] - _sphere_loss(rm, 3)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])
        checked += 1
    assert checked >= 20
