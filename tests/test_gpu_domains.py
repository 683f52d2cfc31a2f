"""Polyhedral domains on the GPU (pc_extract_domain; Section 4.1: a bounded
domain of m half-spaces whose zeros are perturbed only toward the inside)
against the oracle's extract_domain: the box written as half-spaces, the
simplex the paper suggests (Section 5.2) and the cube with one corner cut
off.  Sign vectors and edges bit-exact, coordinates within 1e-6 of the
skeleton's bounding-box diameter; k-cell counts, pruning, invalid input and
context reuse."""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu

DOMAINS = {"simplex": wl.Polytope.simplex, "corner_cut": wl.Polytope.corner_cut}


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


def _tol(dom):
    return 1e-6 * float(np.linalg.norm(dom.X0.max(axis=0) - dom.X0.min(axis=0)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_box_as_halfspaces_equals_the_box(cuda, precision):
    net, box = wl.he_normal_mlp([3, 16, 16, 1], seed=4), wl.Box.cube(3)
    ref = oracle.extract(net, box)
    with cuda(precision=precision) as ex:
        ex.extract_domain(net, wl.Polytope.from_box(box))
        got = _triple(ex)
        ex.extract(net, box)
        box_got = _triple(ex)
    assert_same_complex(got, (ref.X, ref.S, ref.E), coord_tol=1e-6 * 2 * np.sqrt(3), what=f"box domain {precision}")
    assert_same_complex(got, box_got, coord_tol=1e-6 * 2 * np.sqrt(3), what=f"box domain vs box {precision}")


@pytest.mark.parametrize("execution", ["persistent", "stepwise"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", sorted(DOMAINS))
@pytest.mark.parametrize("widths", [[2, 12, 12, 1], [3, 10, 10, 1], [4, 8, 8, 1], [2, 16, 16, 16, 1]])
def test_domain_matches_oracle(cuda, widths, name, precision, execution):
    dom = DOMAINS[name](widths[0])
    for seed in range(2):
        net = wl.he_normal_mlp(widths, seed=900 + seed)
        ref = oracle.extract_domain(net, dom)
        assert ref.status == 0, ref.error
        with cuda(precision=precision, execution=execution) as ex:
            ex.extract_domain(net, dom)
            assert_same_complex(_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(dom),
                                what=f"{name} {widths} seed {seed} {precision} {execution}")


@pytest.mark.parametrize("name", sorted(DOMAINS))
def test_domain_cell_counts(cuda, name):
    net = wl.he_normal_mlp([3, 12, 12, 1], seed=21)
    dom = DOMAINS[name](3)
    ref = oracle.extract_domain(net, dom)
    f_ref, chi_ref = oracle.faces(ref)
    with cuda(precision="mixed") as ex:
        ex.extract_domain(net, dom)
        f, chi = ex.cell_counts()
    assert list(f) == list(f_ref) and chi == chi_ref == 1


@pytest.mark.parametrize("name", sorted(DOMAINS))
def test_domain_pruning_matches_oracle(cuda, name):
    net = wl.he_normal_mlp([3, 10, 10, 10, 1], seed=33)
    dom = DOMAINS[name](3)
    ref = oracle.extract_domain(net, dom, prune=True)
    assert ref.status == 0, ref.error
    with cuda(precision="mixed", prune=True) as ex:
        ex.extract_domain(net, dom)
        assert_same_complex(_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(dom), what=f"{name} pruned")


def test_invalid_domain_is_rejected_and_the_context_stays_usable(cuda):
    from paper_2306_07212_gb300.binding import PcError
    net = wl.he_normal_mlp([2, 8, 8, 1], seed=2)
    dom = wl.Polytope.simplex(2)
    bad = wl.Polytope(dom.A, dom.c, dom.X0 + np.array([0.5, 0.0]), dom.E0)  # a vertex outside
    box = wl.Box.cube(2)
    ref = oracle.extract(net, box)
    with cuda(precision="mixed") as ex:
        with pytest.raises(PcError) as e:
            ex.extract_domain(net, bad)
        assert e.value.status == 1 and "domain" in str(e.value)
        ex.extract(net, box)
        assert_same_complex(_triple(ex), (ref.X, ref.S, ref.E), coord_tol=1e-6 * 2 * np.sqrt(2), what="box after")


def test_one_context_alternates_domains_and_boxes(cuda):
    net = wl.he_normal_mlp([3, 12, 12, 1], seed=8)
    box = wl.Box.cube(3)
    refs = {"box": oracle.extract(net, box)}
    for name, make in DOMAINS.items():
        refs[name] = oracle.extract_domain(net, make(3))
    with cuda(precision="mixed") as ex:
        for name in ["simplex", "box", "corner_cut", "simplex", "box"]:
            if name == "box":
                ex.extract(net, box)
            else:
                ex.extract_domain(net, DOMAINS[name](3))
            r = refs[name]
            assert_same_complex(_triple(ex), (r.X, r.S, r.E), coord_tol=1e-6 * 2 * np.sqrt(3), what=name)
