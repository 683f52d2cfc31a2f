"""Host logic of bench.py's counting sweep, with CUDA and the library faked:
the points it visits, the statistics it reports and a failing point that is
recorded without ending the sweep."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
import paper_2306_07212_gb300 as pkg  # noqa: E402


class _Clock:
    t = 0.0


class _Event:
    def __init__(self, enable_timing=True):
        self.at = None

    def record(self):
        _Clock.t += 2.0
        self.at = _Clock.t

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.at - self.at


class _FakeExtractor:
    opened = []

    def __init__(self, device, precision, execution, max_dim=8):
        self.args = (device, precision, execution)
        self.max_dim = max_dim
        _FakeExtractor.opened.append(self)
        self.closed = False

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.closed = True

    def extract(self, net, box, params=None):
        if net.D > self.max_dim:
            raise RuntimeError(f"input dimension must be in [1, {self.max_dim}]")
        self.net = net

    def counts(self):
        w = self.net.widths[1]
        return {"nV": 100 * self.net.D + w, "nE": 300 * self.net.D + w}

    def vertices(self):
        return np.zeros((self.counts()["nV"], self.net.D))

    def sign_words(self):
        S = (2 * self.net.D + self.net.n_neurons + 31) // 32
        return np.full((S, self.counts()["nV"]), 0x5555555555555555, np.uint64)  # every entry +

    def extract_domain(self, net, dom, params=None):
        assert dom.A.shape[1] == net.D
        self.net = net


@pytest.fixture
def faked(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "memory_allocated", lambda *a, **k: 1 << 20)
    monkeypatch.setattr(torch.cuda, "reset_peak_memory_stats", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "max_memory_allocated", lambda *a, **k: 3 << 20)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(pkg, "Extractor", _FakeExtractor)
    _FakeExtractor.opened = []


def test_dims_spec():
    assert bench._dims("1-4") == [1, 2, 3, 4]
    assert bench._dims("1,2,5") == [1, 2, 5]
    assert bench._dims("2-3,7") == [2, 3, 7]


def test_counting_sweep_points_and_statistics(faked):
    out = bench.run_counting_sweep([1, 3], seeds=2, device=0, precision="mixed", execution="persistent")
    pts = out["points"]
    assert [(p["D"], p["width"]) for p in pts] == [(1, 10), (3, 10), (1, 20), (3, 20), (1, 40), (3, 40)]
    # one fresh context per net, all closed again
    assert len(_FakeExtractor.opened) == 12 and all(e.closed for e in _FakeExtractor.opened)
    assert all(e.args == (0, "mixed", "persistent") for e in _FakeExtractor.opened)
    assert all(("zero_residual_rel" in p) == (p["width"] == 10) for p in pts)
    assert pts[0]["zero_residual_rel"] == 0.0
    p = pts[3]
    assert p["nV"] == [320.0, 0.0] and p["nE"] == [920.0, 0.0]
    assert p["ms"] == [2.0, 0.0] and p["cold_ms"] == [2.0, 0.0]
    assert p["peak_mib"] == [2.0, 0.0]
    assert p["ve_per_s"] == pytest.approx((320 + 920) / 2e-3)


def test_counting_sweep_records_a_failing_point(faked):
    out = bench.run_counting_sweep([8, 11], seeds=1, device=0, precision="mixed", execution="persistent")
    by = {(p["D"], p["width"]): p for p in out["points"]}
    assert "error" in by[(11, 10)] and "[1, 10]" in by[(11, 10)]["error"]
    assert "error" not in by[(8, 40)] and by[(8, 40)]["nV"][0] == 840.0
    assert len(out["points"]) == 6 and np.isfinite(out["seconds"])


def test_width_10_sweep_uses_the_d10_build_above_8(faked):
    out = bench.run_counting_sweep([7, 9, 10], seeds=1, device=0, precision="mixed", execution="persistent",
                                   widths=(10,))
    assert [(p["D"], p["width"]) for p in out["points"]] == [(7, 10), (9, 10), (10, 10)]
    assert [e.max_dim for e in _FakeExtractor.opened] == [8, 10, 10]
    assert all("error" not in p and "zero_residual_rel" in p for p in out["points"])


def test_host_cpu_reports_cores():
    info = bench.host_cpu()
    assert isinstance(info["nproc"], int) and info["nproc"] >= 1


def test_domain_measurement(faked):
    from paper_2306_07212_gb300 import workloads as wl

    class Args:
        precision, execution, warmup, steps = "mixed", "persistent", 3, 4

    class Flush:
        def zero_(self):
            pass

    net = wl.he_normal_mlp([3, 16, 16, 1], seed=0)
    out = bench.run_domain(net, None, Flush(), 0, Args())
    assert out["steps"] == 4 and out["ms_per_step"] == 2.0
    assert (out["n_vertices"], out["n_edges"]) == (316, 916)
    assert out["value"] == pytest.approx((316 + 916) / 2e-3)
    assert "4 vertices, 4 facets" in out["workload"]
    assert len(_FakeExtractor.opened) == 1 and _FakeExtractor.opened[0].closed


def _pack(S):
    """int8 sign vectors (nV, P) -> packed 2-bit words (ceil(P / 32), nV)."""
    nV, P = S.shape
    words = np.zeros(((P + 31) // 32, nV), np.uint64)
    for j in range(P):
        code = np.where(S[:, j] == 1, 1, np.where(S[:, j] == -1, 2, 0)).astype(np.uint64)
        words[j // 32] |= code << np.uint64(2 * (j % 32))
    return words


def test_zero_residual_of_an_exact_complex_and_a_shifted_one():
    import oracle
    from paper_2306_07212_gb300 import workloads as wl
    net, box = wl.counting_sweep_net(3, 10, seed=1)
    r = oracle.extract(net, box)
    words = _pack(r.S)
    assert bench.zero_residual(net, box, r.X, words) < 1e-13
    X = r.X.copy()
    X[5] += 1e-4  # one vertex moved off its zero set
    assert 1e-6 < bench.zero_residual(net, box, X, words) < 1e-3


def test_zero_residual_sees_every_chunk():
    import oracle
    from paper_2306_07212_gb300 import workloads as wl
    net, box = wl.counting_sweep_net(2, 10, seed=2)
    r = oracle.extract(net, box)
    reps = (1 << 20) // r.nV + 2  # more rows than one chunk
    X = np.tile(r.X, (reps, 1))
    words = np.tile(_pack(r.S), (1, reps))
    assert bench.zero_residual(net, box, X, words) < 1e-13
    X[-1] += 1e-4  # a vertex in the last chunk moved off its zero set
    assert bench.zero_residual(net, box, X, words) > 1e-6


def test_neuron_loop_bytes_follow_the_per_step_model():
    """4 V + 8 E + S (3 (8D + 4H + 8W) + 16) + 24 K + 8 P per step (FP32
    values), summed per layer; FP64 values count 8 bytes each."""
    import numpy as np
    from paper_2306_07212_gb300 import workloads as wl
    net = wl.he_normal_mlp([3, 2, 1], seed=0)  # two layers: H = 2, then 1
    stats = np.array([[10, 20, 3, 8, 4, 0, 0, 0],
                      [13, 27, 1, 4, 2, 0, 0, 0],
                      [14, 30, 2, 6, 3, 0, 0, 0]], np.int64)
    W = (2 * 3 + 3 + 31) // 32
    step = lambda V, E, S, K, P, H, zb: zb * V + 8 * E + S * (3 * (8 * 3 + H * zb + 8 * W) + 16) + 24 * K + 8 * P
    got = bench.neuron_loop_bytes(net, stats, "mixed")
    assert got == [step(10, 20, 3, 8, 4, 2, 4) + step(13, 27, 1, 4, 2, 2, 4), step(14, 30, 2, 6, 3, 1, 4)]
    got64 = bench.neuron_loop_bytes(net, stats, "fp64")
    assert got64[1] == step(14, 30, 2, 6, 3, 1, 8)
    gb = bench.gemm_bytes_flops(net, stats, "mixed")
    assert gb[0] == (4 * 10 * (3 + 2) + 8 * W * 10, 2.0 * 10 * 3 * 2)
    assert gb[1] == (4 * 14 * (2 + 1) + 8 * W * 14, 2.0 * 14 * 2 * 1)


def test_loop_roofline_arithmetic():
    r = bench.loop_roofline([2e9, 4e9], [1.0, 3.0], 6000.0, "measured")
    assert r["achieved"] == round(6e9 / 4e-3 / 1e9, 2) and r["bound"] == "hbm"
    assert r["frac"] == round(r["achieved"] / 6000.0, 4) and r["launch_ms_avg"] == 2.0


def test_traffic_is_tied_to_the_kernel_sources():
    sha = bench.kernel_sources_sha16()
    assert len(sha) == 16 and all(ch in "0123456789abcdef" for ch in sha)
    assert sha == bench.kernel_sources_sha16()


def test_captured_traffic_is_reported_only_for_its_sources(monkeypatch):
    key = "k_layer_torus"
    monkeypatch.setitem(bench.KERNEL_DRAM, key, 123)
    monkeypatch.setitem(bench.KERNEL_DRAM, "sources_sha16", bench.kernel_sources_sha16())
    assert bench.kernel_traffic(key, "mixed")["traffic"] == 123
    assert bench.kernel_traffic(key, "fp64")["traffic"] is None  # captured in mixed precision only
    monkeypatch.setitem(bench.KERNEL_DRAM, "sources_sha16", "0" * 16)
    assert bench.kernel_traffic(key, "mixed")["traffic"] is None
