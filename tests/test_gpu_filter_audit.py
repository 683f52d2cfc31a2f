"""Audit of the mixed-precision sign filter (Section 4.2, steps (2) and (4):
the signs decide the combinatorics, so every FP32 sign that could be wrong
must be re-decided in FP64).

The filter re-decides a value z in FP64 at the exact vertex when |z| <= kappa
times its FP32 error estimate (kappa = 12 in production) and writes the FP64
value back, which also makes later interpolated values more accurate.  The
estimate is an rms model, not a worst-case bound, so this test measures, in
the production dynamics, how close to the filter's edge a wrong FP32 sign
comes and whether one gets past it: each extraction runs with kappa = 12 and
an audit band up to 1000 estimates, where every value is also evaluated in
FP64 but only recorded, never written back.  The test asserts

  * that no FP32 sign in the audit band is wrong (the filter missed none);
  * that no sign is undecidable in FP64 (|z| within 1e-12 of its terms);
  * that the audited extraction equals a separate kappa = 1000 extraction and,
    for the 240 random nets, the FP64 oracle's complex;

and prints the largest margin |z| / estimate among the wrong FP32 signs the
filter caught.  Auditing at kappa = 1000 instead of the production dynamics
would understate that margin: at kappa = 3 the net [4, 32, 96, 1] below
gets a sign wrong that a kappa = 1000 run never sees.

The nets: 240 He-normal nets (D = 2, 3, 4; depth 1-4; widths up to 128, up to
~3e5 vertices), the net [4, 32, 96, 1] (7.3e6 vertices) with the tensor-core
and the SIMT layer products, the D=3 torus workload and the D=4 workload's
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


def _run(Extractor, net, box, kappa, audit=0.0, gemm="tensor"):
    with Extractor(precision="mixed", kappa=kappa, kappa_audit=audit, gemm=gemm) as ex:
        ex.extract(net, box)
        c = ex.counts()
        d = ex.diagnostics()
        res = (ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges())
    return res, d


def _audit(Extractor, name, net, box, check_oracle, worst, gemm="tensor"):
    tol = 1e-6 * float(np.linalg.norm(box.hi - box.lo))
    prod, dp = _run(Extractor, net, box, KAPPA, KAPPA_AUDIT, gemm)
    assert dp["undecided"] == 0, (name, dp)
    assert dp["missed"] == 0, (f"{name}: {dp['missed']} wrong FP32 signs beyond kappa {KAPPA} got past the filter "
                               f"(largest at {dp['missed_margin_milli'] / 1000:.2f} estimates)")
    margin = dp["flip_margin_milli"] / 1000.0
    if dp["flips"] and margin > worst[0]:
        worst[:] = [margin, name]
    wide, dw = _run(Extractor, net, box, KAPPA_AUDIT, 0.0, gemm)
    assert dw["undecided"] == 0, (name, dw)
    assert_same_complex(prod, wide, coord_tol=tol, what=f"{name}: kappa {KAPPA} vs {KAPPA_AUDIT}")
    if check_oracle:
        r = oracle.extract(net, box)
        assert r.status == 0, r.error
        assert_same_complex(prod, (r.X, r.S, r.E), coord_tol=tol, what=f"{name}: vs oracle")
    return dp["flips"]


def test_filter_over_random_nets(Extractor):
    worst = [0.0, ""]
    flips = 0
    for name, net, box in _nets():
        flips += _audit(Extractor, name, net, box, check_oracle=True, worst=worst)
    print(f"\nfilter audit, 240 nets: {flips} wrong FP32 signs caught by kappa {KAPPA:g}, none missed up to "
          f"{KAPPA_AUDIT:g} estimates; largest margin {worst[0]:.3f} ({worst[1]})")


@pytest.mark.parametrize("which,gemm", [("torus", "tensor"), ("d4_subbox", "tensor"), ("4-32-96-1", "tensor"),
                                        ("4-32-96-1", "simt")])
def test_filter_on_larger_nets(Extractor, which, gemm):
    if which == "torus":
        net, box = wl.torus_d3()
    elif which == "d4_subbox":
        net, box = wl.precision_d4_subbox()
    else:
        net, box = wl.he_normal_mlp([4, 32, 96, 1], seed=11), wl.Box.cube(4)
    worst = [0.0, ""]
    f = _audit(Extractor, which, net, box, check_oracle=False, worst=worst, gemm=gemm)
    print(f"\nfilter audit, {which} ({gemm} product): {f} wrong FP32 signs caught by kappa {KAPPA:g}, none missed "
          f"up to {KAPPA_AUDIT:g} estimates; largest margin {worst[0]:.3f}")
