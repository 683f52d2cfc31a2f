"""Host checks of a polyhedral domain before pc_extract_domain runs
(pc_check_domain, no GPU needed): simple polytopes with complete skeletons
pass; a vertex outside, a vertex on more than D facets, a missing, doubled
or misplaced edge, a bad index and too few facets are rejected."""
import dataclasses

import numpy as np
import pytest

from paper_2306_07212_gb300 import binding, workloads as wl


@pytest.fixture(scope="module")
def check():
    from paper_2306_07212_gb300 import buildlib
    buildlib.build()
    return binding.check_domain


def _replace(dom, **kw):
    return dataclasses.replace(dom, **{k: np.array(v) for k, v in kw.items()})


@pytest.mark.parametrize("D", range(1, 9))
def test_boxes_simplices_and_cut_cubes_pass(check, D):
    assert check(wl.Polytope.simplex(D))
    assert check(wl.Polytope.from_box(wl.Box.cube(D)))
    assert check(wl.Polytope.corner_cut(D))
    assert check(wl.Polytope.from_box(wl.Box(np.linspace(-2, 0, D), np.linspace(1, 3, D))))


def test_vertex_outside_is_rejected(check):
    dom = wl.Polytope.simplex(3)
    X0 = dom.X0.copy()
    X0[1, 0] += 0.5  # beyond the facet sum(x - lo) <= size
    assert not check(_replace(dom, X0=X0))


def test_vertex_off_its_facets_is_rejected(check):
    dom = wl.Polytope.simplex(2)
    X0 = dom.X0.copy()
    X0[0] += 0.1  # the corner moves inside: it lies on no facet
    assert not check(_replace(dom, X0=X0))


def test_non_simple_vertex_is_rejected(check):
    # square pyramid: the apex lies on four facets in D = 3
    A = np.array([[0, 0, -1], [-1, 0, 1], [1, 0, 1], [0, -1, 1], [0, 1, 1]], float)
    c = np.array([0, 1, 1, 1, 1], float)
    X0 = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0], [0, 0, 1]], float)
    E0 = np.array([[0, 1], [1, 2], [2, 3], [3, 0], [0, 4], [1, 4], [2, 4], [3, 4]], np.int32)
    assert not check(wl.Polytope(A, c, X0, E0))


def test_missing_doubled_and_misplaced_edges_are_rejected(check):
    dom = wl.Polytope.from_box(wl.Box.cube(3))
    assert not check(_replace(dom, E0=dom.E0[1:]))  # two vertices with D - 1 edges
    doubled = dom.E0.copy()
    doubled[1] = doubled[0][::-1]  # edge 0 twice, edge 1 missing
    assert not check(_replace(dom, E0=doubled))
    diag = dom.E0.copy()
    diag[0] = [0, 7]  # a diagonal of the cube lies on no common facet
    assert not check(_replace(dom, E0=diag))
    bad = dom.E0.copy()
    bad[3, 1] = 8  # index out of range
    assert not check(_replace(dom, E0=bad))
    loop = dom.E0.copy()
    loop[3, 1] = loop[3, 0]
    assert not check(_replace(dom, E0=loop))


def test_degenerate_shapes_are_rejected(check):
    dom = wl.Polytope.simplex(3)
    assert not check(_replace(dom, A=dom.A[:3], c=dom.c[:3]))  # m < D + 1
    nan = dom.A.copy()
    nan[0, 0] = np.nan
    assert not check(_replace(dom, A=nan))
    with pytest.raises(ValueError):
        check(_replace(dom, c=dom.c[:2]))  # c does not match A
    with pytest.raises(ValueError):
        check(_replace(dom, E0=dom.E0[:, :1]))
