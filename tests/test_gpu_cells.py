"""k-cell counts on the GPU (pc_cell_counts) against the oracle's counts by
perturbation (Section 4.1), and the Euler characteristic of the subdivided
box (1)."""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("widths", [[2, 8, 8, 1], [3, 8, 8, 1], [4, 6, 6, 1], [3, 16, 16, 1]])
def test_cell_counts_match_oracle(cuda, precision, widths):
    net = wl.he_normal_mlp(widths, seed=1)
    box = wl.Box.cube(widths[0])
    f_ref, chi_ref = oracle.faces(oracle.extract(net, box))
    with cuda(precision=precision) as ex:
        ex.extract(net, box)
        f, chi = ex.cell_counts()
    assert f.tolist() == f_ref.tolist() and chi == chi_ref == 1


def test_torus_regions_and_euler(cuda):
    net, box = wl.torus_d3()
    with cuda(precision="mixed") as ex:
        ex.extract(net, box)
        c = ex.counts()
        f, chi = ex.cell_counts()
    assert f[0] == c["nV"] and f[1] == c["nE"] and chi == 1
    print(f"\ntorus k-cells {f.tolist()}, Euler characteristic {chi}")
