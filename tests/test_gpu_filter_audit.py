"""Audit of the mixed-precision sign filter (Section 4.2, steps (2) and (4):
the signs decide the combinatorics, so every FP32 sign that could be wrong
must be re-decided in FP64).

The filter re-decides a value z in FP64 at the exact vertex when |z| <= kappa
times its FP32 error estimate (kappa = 12 in production).  The estimate is an
rms model, not a worst-case bound, so this test measures how close to the
filter's edge a wrong FP32 sign comes: every extraction runs with the filter
widened to kappa = 1000, and each FP64 re-decision that changes the FP32 sign
records its margin |z| / estimate.  The test asserts

  * that the largest margin over all nets stays below the production kappa
    (so kappa = 12 would have re-decided every sign the FP32 values got wrong);
  * that no sign is undecidable in FP64 (|z| within 1e-12 of its terms);
  * that kappa = 12 and kappa = 1000 give identical complexes, and, where the
    FP64 oracle is quick (the 240 random nets), the oracle's complex.

The nets: 240 He-normal nets (D = 2, 3, 4; depth 1-4; widths up to 128, sized
to stay below ~3e5 vertices), the D=3 torus workload and the D=4 workload's
net on its precision sub-box.
"""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu

KAPPA = 12.0
KAPPA_AUDIT = 1000.0
WIDTHS = {2: (16, 32, 64, 128), 3: (8, 16, 24, 32), 4: (6, 8, 12, 16)}


def _nets():
    out = []
    for s in range(240):
        D = 2 + s % 3
        depth = 1 + (s // 3) % 4
        w = WIDTHS[D][(s // 12) % 4]
        if D == 4 and depth >= 3 and w > 8:
            w = 8
        out.append((f"D{D}-w{w}-d{depth}-s{s}", wl.he_normal_mlp([D] + [w] * depth + [1], seed=5000 + s).rounded_to_fp32(),
                    wl.Box.cube(D)))
    return out


@pytest.fixture(scope="module")
def Extractor():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


def _run(Extractor, net, box, kappa):
    with Extractor(precision="mixed", kappa=kappa) as ex:
        ex.extract(net, box)
        c = ex.counts()
        d = ex.diagnostics()
        res = (ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges())
        filt = int(ex.stats()[:, 5].sum())
    return res, d, filt


def _audit(Extractor, name, net, box, check_oracle, worst):
    tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    wide, dw, fw = _run(Extractor, net, box, KAPPA_AUDIT)
    prod, dp, fp = _run(Extractor, net, box, KAPPA)
    assert dw["undecided"] == 0 and dp["undecided"] == 0, (name, dw, dp)
    margin = dw["flip_margin_milli"] / 1000.0
    if dw["flips"] and margin > worst[0]:
        worst[:] = [margin, name, dw["flips"], fw]
    assert margin < KAPPA, f"{name}: an FP32 sign was wrong at {margin:.2f} x its error estimate (kappa {KAPPA})"
    assert_same_complex(prod, wide, coord_tol=tol, what=f"{name}: kappa {KAPPA} vs {KAPPA_AUDIT}")
    if check_oracle:
        r = oracle.extract(net, box)
        assert r.status == 0, r.error
        assert_same_complex(prod, (r.X, r.S, r.E), coord_tol=tol, what=f"{name}: vs oracle")
    return dw["flips"], fw


def test_filter_margin_over_random_nets(Extractor):
    worst = [0.0, "", 0, 0]
    flips = refiltered = 0
    for k, (name, net, box) in enumerate(_nets()):
        f, r = _audit(Extractor, name, net, box, check_oracle=True, worst=worst)
        flips += f
        refiltered += r
    print(f"\nfilter audit, 240 nets: {flips} wrong FP32 signs among {refiltered} re-decisions at kappa "
          f"{KAPPA_AUDIT:g}; largest margin {worst[0]:.3f} ({worst[1]}); production kappa {KAPPA:g}")


@pytest.mark.parametrize("which", ["torus", "d4_subbox"])
def test_filter_margin_on_the_workloads(Extractor, which):
    net, box = wl.torus_d3() if which == "torus" else wl.precision_d4_subbox()
    worst = [0.0, "", 0, 0]
    f, r = _audit(Extractor, which, net, box, check_oracle=False, worst=worst)
    print(f"\nfilter audit, {which}: {f} wrong FP32 signs among {r} re-decisions at kappa {KAPPA_AUDIT:g}; "
          f"largest margin {worst[0]:.3f}")
