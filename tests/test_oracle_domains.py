"""Pins of the oracle on general polyhedral domains (Section 4.1: a bounded
domain given by m affine half-spaces, boundary zeros perturbed only toward
the inside), e.g. the simplex the paper suggests in place of the box:

  * the box written as 2D half-spaces with its corners and axis edges gives
    the box extraction bit for bit;
  * on tiny nets the simplex-domain extraction equals the complex built from
    the definition (brute force) on the same domain;
  * the subdivided simplex has Euler characteristic 1;
  * a line arrangement in a triangle: V = 3 + 2 n_in + I, E = 3 + 3 n_in + 2 I
    (n_in lines crossing the open triangle, I crossings inside it).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex


@pytest.mark.parametrize("widths,seed", [([2, 8, 8, 1], 0), ([3, 6, 6, 1], 1), ([2, 12, 1], 2), ([4, 5, 5, 1], 3)])
def test_box_as_halfspaces_is_the_box_extraction(widths, seed):
    net = wl.he_normal_mlp(widths, seed=seed)
    box = wl.Box.cube(widths[0])
    a = oracle.extract(net, box)
    b = oracle.extract_domain(net, wl.Polytope.from_box(box))
    assert a.status == 0 and b.status == 0
    assert np.array_equal(a.X, b.X) and np.array_equal(a.S, b.S) and np.array_equal(a.E, b.E)


@pytest.mark.parametrize("widths", [[2, 4, 3, 1], [2, 3, 3, 3, 1], [3, 4, 3, 1], [3, 3, 3, 3, 1], [2, 6, 1]])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_simplex_matches_brute_force(widths, seed):
    net = wl.he_normal_mlp(widths, seed=300 + seed)
    dom = wl.Polytope.simplex(widths[0])
    r = oracle.extract_domain(net, dom)
    b = oracle.brute_domain(net, dom, tol=1e-9)
    assert r.status == 0 and b.status == 0, (r.error, b.error)
    assert_same_complex((r.X, r.S, r.E), (b.X, b.S, b.E), coord_tol=1e-9, what=f"simplex {widths} seed {seed}")


@pytest.mark.parametrize("widths", [[2, 10, 10, 1], [3, 8, 8, 1], [4, 6, 6, 1]])
def test_simplex_euler_characteristic(widths):
    r = oracle.extract_domain(wl.he_normal_mlp(widths, seed=5), wl.Polytope.simplex(widths[0]))
    f, chi = oracle.faces(r)
    assert r.status == 0 and chi == 1 and f[0] == r.nV and f[1] == len(r.E)


@pytest.mark.parametrize("n", [1, 4, 9, 20])
@pytest.mark.parametrize("seed", [0, 1])
def test_line_arrangement_in_a_triangle(n, seed):
    net = wl.he_normal_mlp([2, n], seed=seed, bias_var=0.25)
    dom = wl.Polytope.simplex(2)
    r = oracle.extract_domain(net, dom)
    assert r.status == 0
    W, b = net.W[0], net.b[0]
    vals = dom.X0 @ W.T + b
    n_in = int(((vals.max(axis=0) > 0) & (vals.min(axis=0) < 0)).sum())
    I = 0
    for i, j in itertools.combinations(range(n), 2):
        x = np.linalg.solve(np.stack([W[i], W[j]]), -np.array([b[i], b[j]]))
        if np.all(dom.c - dom.A @ x > 0):
            I += 1
    assert r.nV == 3 + 2 * n_in + I
    assert len(r.E) == 3 + 3 * n_in + 2 * I


# --- a domain that is neither a box nor a simplex ---------------------------

@pytest.mark.parametrize("widths", [[2, 4, 3, 1], [2, 3, 3, 3, 1], [3, 4, 3, 1], [3, 3, 3, 1], [2, 6, 1]])
@pytest.mark.parametrize("seed", [0, 1])
def test_corner_cut_cube_matches_brute_force(widths, seed):
    net = wl.he_normal_mlp(widths, seed=700 + seed)
    dom = wl.Polytope.corner_cut(widths[0])
    r = oracle.extract_domain(net, dom)
    b = oracle.brute_domain(net, dom, tol=1e-9)
    assert r.status == 0 and b.status == 0, (r.error, b.error)
    assert_same_complex((r.X, r.S, r.E), (b.X, b.S, b.E), coord_tol=1e-9, what=f"corner cut {widths} seed {seed}")


@pytest.mark.parametrize("D", [1, 2, 3, 4])
def test_corner_cut_skeleton_and_euler_characteristic(D):
    dom = wl.Polytope.corner_cut(D)
    assert len(dom.X0) == 2 ** D - 1 + D
    assert len(dom.E0) == D * 2 ** (D - 1) + D * (D - 1) // 2
    assert np.all(np.bincount(dom.E0.ravel(), minlength=len(dom.X0)) == D)
    r = oracle.extract_domain(wl.he_normal_mlp([D, 8, 8, 1], seed=D), dom)
    f, chi = oracle.faces(r)
    assert r.status == 0 and chi == 1


@pytest.mark.parametrize("name", ["simplex", "corner_cut"])
@pytest.mark.parametrize("widths", [[4, 3, 2, 1], [5, 3, 1], [6, 2, 2, 1]])
def test_higher_dimensional_domains_match_brute_force(name, widths):
    net = wl.he_normal_mlp(widths, seed=61)
    dom = getattr(wl.Polytope, name)(widths[0])
    r = oracle.extract_domain(net, dom)
    b = oracle.brute_domain(net, dom, tol=1e-9)
    assert r.status == 0 and b.status == 0, (r.error, b.error)
    assert_same_complex((r.X, r.S, r.E), (b.X, b.S, b.E), coord_tol=1e-9, what=f"{name} {widths}")
