"""Serving (pc_server_*): continuous admission of extraction requests.

Each result computed inside a mix of concurrently running requests must be
the same as the same request run alone through pc_extract; oversize requests
are rejected with PC_ERR_TOO_LARGE; admission keeps the summed memory
estimates within the budget; one slot is a FIFO path.
"""
import time

import numpy as np
import pytest

from paper_2306_07212_gb300 import workloads as wl
from _util import assert_same_complex, unpack_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_07212_gb300 import binding
    return binding


def _mix(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        D = int(rng.choice([2, 3]))
        depth = int(rng.integers(2, 4))
        width = int(rng.choice([8, 12, 16]))
        out.append(wl.random_mlp(D, depth, width, seed=500 + k))
    return out


def test_each_result_same_alone_and_in_the_mix(gpu):
    reqs = _mix(16)
    with gpu.Server(max_slots=4, precision="mixed", keep_outputs=True) as srv:
        ids = [srv.submit(net, box) for net, box in reqs]
        srv.wait_all(300)
        mixed = []
        for rid in ids:
            st, r = srv.poll(rid)
            assert st == 0 and r.status == 0, (r.status, srv.error(rid))
            mixed.append(srv.outputs(rid))
        slots = {srv.poll(rid)[1].slot for rid in ids}
    assert len(slots) > 1, "requests should spread over several slots"
    with gpu.Extractor(precision="mixed", execution="stepwise", polish=0) as ex:
        for (net, box), (X, SIG, E) in zip(reqs, mixed):
            ex.extract(net, box)
            c = ex.counts()
            alone = (ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges())
            got = (X, unpack_codes(SIG, c["P"]), E)
            assert_same_complex(got, alone, coord_tol=1e-12, what=f"{net.widths}")


def test_stream_requests_same_alone_and_in_the_mix(gpu):
    """Requests of the configured serving stream itself (D up to 4, depth 2-6,
    widths 16-128), the first 40 whose memory estimate is at most 2 GiB
    (each takes at most ~20 ms): the same complex in an 8-slot mix as alone."""
    reqs = [r for r in wl.serving_stream(300) if gpu.estimate_bytes(r.net) <= 2 << 30][:40]
    assert max(r.net.D for r in reqs) == 4 and max(max(r.net.widths[1:]) for r in reqs) == 128
    with gpu.Server(max_slots=8, precision="mixed", keep_outputs=True) as srv:
        ids = [srv.submit(r.net, r.box) for r in reqs]
        srv.wait_all(600)
        mixed = []
        for rid in ids:
            st, res = srv.poll(rid)
            assert st == 0 and res.status == 0, (res.status, srv.error(rid))
            mixed.append(srv.outputs(rid))
    with gpu.Extractor(precision="mixed", execution="stepwise", polish=0) as ex:
        for r, (X, SIG, E) in zip(reqs, mixed):
            ex.extract(r.net, r.box)
            c = ex.counts()
            alone = (ex.vertices(), unpack_codes(ex.sign_words(), c["P"]), ex.edges())
            got = (X, unpack_codes(SIG, c["P"]), E)
            assert_same_complex(got, alone, coord_tol=1e-12, what=f"stream request {r.rid} {r.net.widths}")


def test_oversize_request_is_rejected(gpu):
    net, box = wl.random_mlp(4, 6, 128, seed=1)
    with gpu.Server(max_slots=2, request_max_bytes=1 << 30) as srv:
        rid = srv.submit(net, box)
        st, r = srv.poll(rid)
        assert st == 0 and r.status == 6 and r.slot == -1


def test_admission_respects_the_memory_budget(gpu):
    reqs = [wl.random_mlp(3, 2, 16, seed=900 + k) for k in range(12)]
    one = gpu.estimate_bytes(reqs[0][0])
    budget = int(2.5 * one)
    with gpu.Server(max_slots=8, mem_budget_bytes=budget, request_max_bytes=budget) as srv:
        ids = [srv.submit(net, box) for net, box in reqs]
        srv.wait_all(300)
        assert all(srv.poll(i)[1].status == 0 for i in ids)
        assert srv.stats()["peak_bytes"] <= budget


def test_single_slot_is_fifo(gpu):
    reqs = _mix(6, seed=3)
    with gpu.Server(max_slots=1) as srv:
        ids = [srv.submit(net, box) for net, box in reqs]
        srv.wait_all(300)
        res = [srv.poll(i)[1] for i in ids]
    starts = [r.start_s for r in res]
    assert starts == sorted(starts)
    for a, b in zip(res, res[1:]):
        assert b.start_s >= a.finish_s - 1e-6
