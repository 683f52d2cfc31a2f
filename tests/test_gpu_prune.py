"""Pruning during edge subdivision on the GPU (pc_options.prune, Section
5.4.2) against the oracle's pruned extraction: the same vertices (sign
vectors), edges and coordinates; the level set of the output neuron equals
the full extraction's."""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("D,widths,seed", [(2, [2, 12, 12, 12, 1], 3), (3, [3, 16, 16, 1], 0),
                                           (3, [3, 8, 8, 8, 1], 5), (4, [4, 8, 8, 1], 2)])
def test_pruned_extraction_matches_oracle(cuda, precision, D, widths, seed):
    net = wl.he_normal_mlp(widths, seed=seed)
    box = wl.Box.cube(D)
    ref = oracle.extract(net, box, prune=True)
    assert ref.status == 0
    tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    with cuda(precision=precision, prune=True) as ex:
        ex.extract(net, box)
        assert_same_complex(_triple(ex), (ref.X, ref.S, ref.E), coord_tol=tol, what=f"{widths} pruned {precision}")
    full = oracle.extract(net, box)
    assert len(ref.E) <= len(full.E)


def test_pruned_torus_keeps_the_level_set(cuda):
    net, box = wl.torus_d3()
    with cuda(precision="mixed", prune=True) as ex:
        ex.extract(net, box)
        X, S, E = _triple(ex)
    with cuda(precision="mixed") as ex:
        ex.extract(net, box)
        Xf, Sf, Ef = _triple(ex)
    on, onf = S[:, -1] == 0, Sf[:, -1] == 0
    key = lambda A: {r.tobytes() for r in A}
    assert key(S[on]) == key(Sf[onf])
    assert len(X) < 0.5 * len(Xf) and len(E) < 0.5 * len(Ef)
    print(f"\ntorus pruned: {len(X)} V {len(E)} E (full {len(Xf)} V {len(Ef)} E, level set {int(on.sum())} V)")


def test_prune_rejects_keep_tape(cuda):
    from paper_2306_07212_gb300.binding import PcError
    with pytest.raises(PcError):
        cuda(prune=True, keep_tape=True)
