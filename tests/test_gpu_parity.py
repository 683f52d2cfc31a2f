"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Sign vectors and edge sets must be bit-identical after canonical ordering;
coordinates within 1e-6 of the box diameter (2*sqrt(D) for [-1,1]^D).
"""
import numpy as np
import pytest

import oracle
from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, canon, unpack_codes, entry_values

pytestmark = pytest.mark.gpu


def _gpu_triple(ex):
    c = ex.counts()
    return ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges()


def _tol(box):
    return 1e-6 * float(np.linalg.norm(box.hi - box.lo))


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import Extractor
    return Extractor


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("execution", ["persistent", "stepwise"])
def test_small_d2_config(cuda, precision, execution):
    net, box = wl.small_d2()
    ref = oracle.extract(net, box)
    with cuda(precision=precision, execution=execution) as ex:
        ex.extract(net, box)
        assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box),
                            what=f"2-8-8-1 {precision} {execution}")
        st = ex.stats()
        assert np.array_equal(st[:, 2], ref.stats[:, 0]), "splits per neuron"
        assert np.array_equal(st[:, 4], ref.stats[:, 2]), "paired faces per neuron"


SWEEP = [(1, [1, 8, 8, 1]), (1, [1, 16, 16, 16, 1]), (2, [2, 4, 1]), (2, [2, 16, 16, 1]),
         (2, [2, 12, 12, 12, 12, 1]), (3, [3, 8, 8, 1]), (3, [3, 16, 16, 1]), (3, [3, 6, 6, 6, 6, 2]),
         (4, [4, 8, 8, 1]), (4, [4, 12, 12, 1]), (2, [2, 40, 1]), (3, [3, 2, 2, 1])]


@pytest.mark.parametrize("D,widths", SWEEP)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_random_sweep(cuda, D, widths, precision):
    for seed in range(3):
        net = wl.he_normal_mlp(widths, seed=1000 + seed)
        box = wl.Box.cube(D)
        ref = oracle.extract(net, box)
        assert ref.status == 0
        with cuda(precision=precision) as ex:
            ex.extract(net, box)
            assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box),
                                what=f"{widths} seed {seed} {precision}")


@pytest.mark.parametrize("execution", ["persistent", "stepwise"])
def test_capacity_growth_replays_to_same_result(cuda, execution):
    net = wl.he_normal_mlp([3, 16, 16, 16, 1], seed=4)
    box = wl.Box.cube(3)
    ref = oracle.extract(net, box)
    with cuda(precision="mixed", execution=execution, init_vcap=64, init_ecap=64) as ex:
        ex.extract(net, box)
        assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box), what="growth")
    with cuda(precision="mixed", execution=execution) as ex:
        ex.extract(net, box)
        assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box), what="no growth")


def test_context_reuse_across_networks(cuda):
    nets = [wl.he_normal_mlp(w, seed=s) for s, w in enumerate([[2, 8, 1], [3, 16, 16, 1], [2, 8, 8, 8, 1]])]
    with cuda(precision="mixed") as ex:
        for net in nets + nets[::-1]:
            box = wl.Box.cube(net.D)
            ref = oracle.extract(net, box)
            ex.extract(net, box)
            assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box), what="reuse")


def test_diff_config_d3(cuda):
    net, box = wl.diff_d3()
    ref = oracle.extract(net, box)
    with cuda(precision="mixed") as ex:
        ex.extract(net, box)
        assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box), what="3-32-32-32-1")


def test_torus_config_full_size(cuda):
    """The D=3 torus network at full size (~3e5 vertices, ~9e5 edges)."""
    net, box = wl.torus_d3()
    ref = oracle.extract(net, box)
    assert ref.status == 0
    with cuda(precision="mixed") as ex:
        ex.extract(net, box)
        got = _gpu_triple(ex)
        assert_same_complex(got, (ref.X, ref.S, ref.E), coord_tol=_tol(box), what="torus")
        # the paper's validation (Section 5.1.1): zero entries evaluate to ~0
        vals = entry_values(net, box, got[0])
        assert np.max(np.abs(vals[got[1] == 0])) < 1e-6


def test_zero_residual_and_degree_any_size(cuda):
    """Properties that hold at any size, checked on a larger D=4 net."""
    net = wl.he_normal_mlp([4, 24, 24, 1], seed=3)
    box = wl.Box.cube(4)
    with cuda(precision="mixed") as ex:
        ex.extract(net, box)
        X, S, E = _gpu_triple(ex)
    D, m = 4, 8
    assert np.all((S == 0).sum(axis=1) == D)
    deg = np.bincount(E.ravel(), minlength=len(X))
    assert np.array_equal(deg, 2 * D - (S[:, :m] == 0).sum(axis=1))
    vals = entry_values(net, box, X)
    assert np.max(np.abs(vals[S == 0])) < 1e-6
    # away from zero the recorded sign is the sign at the coordinates (within
    # 1e-5 of zero the FP32-accurate coordinates of unpolished vertices decide
    # nothing: the recorded sign was decided at the exact vertex)
    sure = (S != 0) & (np.abs(vals) > 1e-5)
    assert np.all(np.sign(vals[sure]) == S[sure])


def test_context_keeps_its_buffer_shape_through_growth(cuda):
    """A context that grew its buffers while running a narrow network must
    still fit a wider network that it had sized for before."""
    wide = wl.he_normal_mlp([2, 96, 96, 1], seed=31)
    narrow = wl.he_normal_mlp([2, 8, 8, 8, 1], seed=32)
    box = wl.Box.cube(2)
    with cuda(precision="mixed", init_vcap=64, init_ecap=64) as ex:
        for net in (wide, narrow, wide):
            ref = oracle.extract(net, box)
            ex.extract(net, box)
            assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box),
                                what=f"sequence {net.widths}")


@pytest.mark.parametrize("widths", [[3, 64, 64, 64, 1], [2, 16, 128, 40, 8, 1], [4, 32, 96, 1]])
@pytest.mark.parametrize("gemm", ["tensor", "tensor3x"])
def test_tensor_core_product_matches_simt_and_oracle(cuda, widths, gemm):
    """The tcgen05 layer products (three-piece split, the default, and
    3xTF32) and the SIMT FP32 product give the oracle's complex; their
    final-layer values agree to FP32 accuracy."""
    net = wl.he_normal_mlp(widths, seed=11)
    box = wl.Box.cube(widths[0])
    ref = oracle.extract(net, box)
    with cuda(precision="mixed", gemm=gemm) as a, cuda(precision="mixed", gemm="simt") as b:
        a.extract(net, box)
        b.extract(net, box)
        for ex, name in ((a, gemm), (b, "simt")):
            assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box), what=f"{widths} {name}")
        assert a.diagnostics()["launches"] > 0
        va, vb = a.values(), b.values()
        assert va.shape == vb.shape
        # vertices are numbered in creation order, which follows the
        # (unordered) edge emission: match them by sign vector
        ka = {r.tobytes(): k for k, r in enumerate(np.ascontiguousarray(a.sign_words().T))}
        perm = np.array([ka[r.tobytes()] for r in np.ascontiguousarray(b.sign_words().T)])
        scale = max(1.0, float(np.max(np.abs(vb))))
        assert float(np.max(np.abs(va[perm] - vb))) <= 1e-4 * scale


@pytest.mark.parametrize("D,widths", [(2, [2, 12, 12, 12, 12, 1]), (3, [3, 16, 16, 1]), (4, [4, 12, 12, 1])])
@pytest.mark.parametrize("execution", ["persistent", "stepwise"])
def test_inline_and_deferred_pairing_agree_with_oracle(cuda, D, widths, execution):
    """Step 5 both ways: fingerprint pairing checked after the extraction
    (default) and pairing verified before it is made."""
    net = wl.he_normal_mlp(widths, seed=77)
    box = wl.Box.cube(D)
    ref = oracle.extract(net, box)
    for pairing in ("deferred", "inline"):
        with cuda(precision="mixed", execution=execution, pairing=pairing) as ex:
            ex.extract(net, box)
            assert_same_complex(_gpu_triple(ex), (ref.X, ref.S, ref.E), coord_tol=_tol(box),
                                what=f"{widths} {pairing} {execution}")
            assert ex.diagnostics()["reruns"] == 0


def test_mixed_result_does_not_depend_on_the_launch_grid(cuda):
    """The persistent kernel (two CTAs per SM) and the stepwise kernels (grids
    sized to the edge capacity, here from the default and from a large initial
    capacity) number and batch the new vertices differently; every value, FP64
    re-decision and polish step is still computed per vertex in a fixed order,
    so the complex is the same, coordinates to the last bits (a served request
    must equal the same request run alone)."""
    net, box = wl.torus_d3()
    runs = []
    for execution, vcap, ecap in (("persistent", 0, 0), ("stepwise", 0, 0), ("stepwise", 1 << 20, 1 << 22)):
        with cuda(precision="mixed", execution=execution, init_vcap=vcap, init_ecap=ecap) as ex:
            ex.extract(net, box)
            runs.append(((execution, vcap), _gpu_triple(ex)))
    (name0, ref), rest = runs[0], runs[1:]
    for name, r in rest:
        assert_same_complex(r, ref, coord_tol=1e-12, what=f"{name} against {name0}")
