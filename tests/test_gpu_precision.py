"""Precision study on the D=4 network 4-128x3-1 (He-normal, rounded to FP32).

The three precision modes of the library run on the same network and box as
the FP64 oracle, and the test reports (and for the exact modes asserts) the
combinatorial mismatches and coordinate errors:

  * FP64 throughout, and mixed precision (FP32 values from the tensor-core
    product, FP64 re-decision of every sign within kappa of its FP32 error
    scale, FP64 crossing parameters, float-float polish) with the default
    three-piece product and with the 3xTF32 product: identical sign vectors
    and edges, coordinates within 1e-6 of the box diameter;
  * FP32 values and FP32 sign decisions: reported only (its combinatorics
    may differ where a value is within its FP32 error of zero).

The box is the centred sub-box [-0.02, 0.02]^4 (about 2e5 vertices), which
the oracle finishes in seconds; the full box is beyond it.
"""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import unpack_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def study():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    net, box = wl.precision_d4_subbox()
    ref = oracle.extract(net, box)
    assert ref.status == 0
    return Extractor, net, box, ref


def _compare(ex, ref, box):
    c = ex.counts()
    X = ex.vertices()
    S = unpack_codes(ex.sign_words(), c["P"])
    E = ex.edges()
    rk = {r.astype(np.int8).tobytes(): i for i, r in enumerate(ref.S)}
    gk = [r.astype(np.int8).tobytes() for r in S]
    idx = np.array([rk.get(k, -1) for k in gk])
    matched = idx >= 0
    extra_v = int((~matched).sum())
    missing_v = len(ref.S) - len(set(idx[matched].tolist()))

    def edge_keys(Sv, Ev):
        keys = [r.astype(np.int8).tobytes() for r in Sv]
        return {tuple(sorted((keys[a], keys[b]))) for a, b in np.asarray(Ev)}

    eg, er = edge_keys(S, E), edge_keys(ref.S, ref.E)
    diam = float(np.linalg.norm(box.hi - box.lo))
    err = np.abs(X[matched] - ref.X[idx[matched]]).max(axis=1) / diam if matched.any() else np.zeros(1)
    return {"nV": len(X), "nE": len(E), "extra_v": extra_v, "missing_v": missing_v,
            "edge_symdiff": len(eg ^ er), "max_err": float(err.max()), "median_err": float(np.median(err)),
            "filtered": int(ex.stats()[:, 5].sum()), "undecided": ex.diagnostics()["undecided"]}


@pytest.mark.parametrize("precision,gemm", [("fp64", "tensor"), ("mixed", "tensor"), ("mixed", "tensor3x"),
                                            ("fp32", "tensor")])
def test_precision_modes_against_oracle(study, precision, gemm):
    Extractor, net, box, ref = study
    with Extractor(precision=precision, gemm=gemm) as ex:
        ex.extract(net, box)
        r = _compare(ex, ref, box)
    print(f"\nprecision study 4-128x3-1 on [-0.02,0.02]^4 ({len(ref.S)} V, {len(ref.E)} E): "
          f"{precision}/{gemm}: {r}")
    if precision != "fp32":
        assert r["extra_v"] == 0 and r["missing_v"] == 0 and r["edge_symdiff"] == 0, r
        assert r["max_err"] <= 1e-6, r
