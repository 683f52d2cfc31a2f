"""Pins of the oracle's pruning during edge subdivision (Section 5.4.2):
after each layer but the last, edges whose vertices have the same signs
w.r.t. all future neurons are dropped, with the vertices left without an
edge.  What must hold, whatever the network:

  * the pruned result is a sub-complex of the full one (same sign vectors,
    same coordinates, same edges);
  * the level set -- the vertices on the output neuron's zero set and the
    edges between them -- is exactly the full extraction's, and on tiny
    nets exactly that of the brute-force complex built from the definition;
  * a network whose output has no zero in the box prunes to nothing;
  * pruning never grows a layer's vertex or edge count.
"""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl


def _keys(S):
    return [r.astype(np.int8).tobytes() for r in S]


def _level_set(r, out_entry):
    """{sign vector: coordinates} of the output zero set, and its edges as
    pairs of sign vectors."""
    on = r.S[:, out_entry] == 0
    keys = _keys(r.S)
    verts = {keys[v]: r.X[v] for v in np.nonzero(on)[0]}
    edges = {tuple(sorted((keys[a], keys[b]))) for a, b in r.E if on[a] and on[b]}
    return verts, edges


def _assert_same_level_set(a, b, out_entry, tol, what):
    va, ea = _level_set(a, out_entry)
    vb, eb = _level_set(b, out_entry)
    assert set(va) == set(vb), f"{what}: level-set vertices differ ({len(va)} vs {len(vb)})"
    for k in va:
        assert np.max(np.abs(va[k] - vb[k])) <= tol, what
    assert ea == eb, f"{what}: level-set edges differ ({len(ea)} vs {len(eb)})"


NETS = [(2, [2, 12, 12, 12, 1], 3), (3, [3, 16, 16, 1], 0), (3, [3, 8, 8, 8, 1], 5), (4, [4, 8, 8, 1], 2),
        (2, [2, 24, 1], 7)]


@pytest.mark.parametrize("D,widths,seed", NETS)
def test_pruned_is_a_subcomplex_with_the_same_level_set(D, widths, seed):
    net = wl.he_normal_mlp(widths, seed=seed)
    box = wl.Box.cube(D)
    full = oracle.extract(net, box)
    pr = oracle.extract(net, box, prune=True)
    assert full.status == 0 and pr.status == 0
    fk = {k: i for i, k in enumerate(_keys(full.S))}
    pk = _keys(pr.S)
    idx = np.array([fk[k] for k in pk], dtype=np.int64)  # KeyError: a vertex the full run lacks
    if len(idx):
        assert np.max(np.abs(pr.X - full.X[idx])) == 0.0
    fe = {tuple(sorted(e)) for e in full.E.tolist()}
    assert all(tuple(sorted((idx[a], idx[b]))) in fe for a, b in pr.E.tolist())
    out_entry = 2 * D + net.n_neurons - 1
    _assert_same_level_set(full, pr, out_entry, 0.0, f"{widths}")
    lf, lp = oracle.layer_counts(full), oracle.layer_counts(pr)
    assert np.all(lp <= lf)


@pytest.mark.parametrize("D,widths", [(2, [2, 4, 3, 1]), (2, [2, 3, 3, 3, 1]), (3, [3, 4, 3, 1]),
                                      (3, [3, 3, 3, 3, 1]), (4, [4, 3, 2, 1]), (5, [5, 2, 2, 1]),
                                      (6, [6, 2, 2, 1])])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pruned_level_set_matches_brute_force(D, widths, seed):
    net = wl.he_normal_mlp(widths, seed=200 + seed)
    box = wl.Box.cube(D)
    pr = oracle.extract(net, box, prune=True)
    b = oracle.brute(net, box, tol=1e-9)
    assert pr.status == 0 and b.status == 0
    _assert_same_level_set(b, pr, 2 * D + net.n_neurons - 1, 1e-9, f"{widths} seed {seed}")


def test_no_level_set_prunes_to_nothing():
    net = wl.he_normal_mlp([3, 8, 8, 1], seed=4)
    net.b[-1][:] = 100.0  # the output is positive on the whole box
    box = wl.Box.cube(3)
    pr = oracle.extract(net, box, prune=True)
    assert pr.status == 0 and pr.nV == 0 and len(pr.E) == 0
    full = oracle.extract(net, box)
    assert not np.any(full.S[:, -1] == 0)


def test_pruning_removes_most_of_a_typical_complex():
    net = wl.he_normal_mlp([3, 16, 16, 1], seed=0)
    box = wl.Box.cube(3)
    lf = oracle.layer_counts(oracle.extract(net, box))
    lp = oracle.layer_counts(oracle.extract(net, box, prune=True))
    assert lp[-1, 0] < 0.5 * lf[-1, 0] and lp[-1, 1] < 0.5 * lf[-1, 1]
