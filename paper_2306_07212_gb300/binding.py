"""Thin Python binding of libpc (include/pc.h) over ctypes.

Argument marshalling only: every step of the extraction runs in the CUDA
library.  PyTorch is used for device memory (the library's buffers come from
torch's caching allocator through pc_set_allocator) and for streams.  There is
no CPU fallback: if the compiled library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from .buildlib import LIB, LIB_D10

PC_OK = 0
STATUS_NAMES = {0: "PC_OK", 1: "PC_ERR_INVALID", 2: "PC_ERR_OOM", 3: "PC_ERR_CUDA",
                4: "PC_ERR_DEGENERATE", 5: "PC_ERR_PAIRING", 6: "PC_ERR_TOO_LARGE",
                7: "PC_ERR_TIMEOUT", 8: "PC_ERR_NO_TAPE", 9: "PC_PENDING"}
PRECISION = {"fp32": 0, "mixed": 1, "fp64": 2}
GEMM = {"tensor": 0, "simt": 1, "tensor3x": 2}
PAIRING = {"deferred": 0, "inline": 1}
EXEC = {"persistent": 0, "stepwise": 1}

# Every symbol include/pc.h declares (checked by the tests).
EXPORTS = ["pc_default_options", "pc_create", "pc_destroy", "pc_set_allocator", "pc_extract",
           "pc_counts", "pc_vertices", "pc_edges", "pc_signvectors", "pc_stats", "pc_backward",
           "pc_diagnostics", "pc_kernel_times", "pc_error_estimates", "pc_values", "pc_extract_noalloc",
           "pc_estimate_bytes", "pc_server_default_options", "pc_server_create", "pc_server_submit",
           "pc_server_poll", "pc_server_error", "pc_server_wait_all", "pc_server_outputs", "pc_server_release", "pc_server_stats",
           "pc_server_destroy", "pc_last_error", "pc_cell_counts", "pc_extract_domain", "pc_check_domain",
           "pc_build_poset", "pc_poset_level"]


class PcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ServerOptions(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("precision", ctypes.c_int), ("exec", ctypes.c_int),
                ("polish", ctypes.c_int), ("keep_outputs", ctypes.c_int),
                ("mem_budget_bytes", ctypes.c_int64), ("request_max_bytes", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_vertices", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("arrival_s", ctypes.c_double), ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double),
                ("est_bytes", ctypes.c_int64), ("slot", ctypes.c_int), ("held_bytes", ctypes.c_int64)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("exec", ctypes.c_int), ("keep_tape", ctypes.c_int),
                ("strict", ctypes.c_int), ("init_vcap", ctypes.c_int64), ("init_ecap", ctypes.c_int64),
                ("mem_budget_bytes", ctypes.c_int64), ("filter_kappa", ctypes.c_double),
                ("polish", ctypes.c_int), ("polish_tol", ctypes.c_double), ("timers", ctypes.c_int),
                ("gemm", ctypes.c_int), ("pairing", ctypes.c_int), ("canonical", ctypes.c_int),
                ("prune", ctypes.c_int), ("debug_barrier_timeout", ctypes.c_int),
                ("filter_kappa_audit", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_libs = {}
_lock = threading.Lock()


def load_library(path: str = LIB):
    """Loads libpc.so (or another build of it, e.g. LIB_D10); raises if it
    has not been built."""
    with _lock:
        if path in _libs:
            return _libs[path]
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, i64p, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
        lib.pc_default_options.argtypes = [ctypes.POINTER(Options)]
        lib.pc_default_options.restype = None
        lib.pc_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(Options)]
        lib.pc_destroy.argtypes = [vp]
        lib.pc_set_allocator.argtypes = [vp, ALLOC_FN, FREE_FN, vp]
        lib.pc_extract.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp]
        lib.pc_counts.argtypes = [vp, i64p, i64p, i32p, i32p, i32p]
        lib.pc_vertices.argtypes = [vp, ctypes.POINTER(vp), i64p, vp]
        lib.pc_edges.argtypes = [vp, ctypes.POINTER(vp), i64p, vp]
        lib.pc_signvectors.argtypes = [vp, ctypes.POINTER(vp), i64p, vp]
        lib.pc_stats.argtypes = [vp, i64p, ctypes.c_int]
        lib.pc_backward.argtypes = [vp, vp, vp, vp]
        lib.pc_diagnostics.argtypes = [vp, i64p, ctypes.c_int]
        lib.pc_error_estimates.argtypes = [vp, vp, vp]
        lib.pc_values.argtypes = [vp, vp]
        lib.pc_estimate_bytes.argtypes = [ctypes.c_int, vp]
        lib.pc_estimate_bytes.restype = ctypes.c_int64
        lib.pc_server_default_options.argtypes = [ctypes.POINTER(ServerOptions)]
        lib.pc_server_default_options.restype = None
        lib.pc_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ServerOptions)]
        lib.pc_server_submit.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.pc_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
        lib.pc_server_wait_all.argtypes = [vp, ctypes.c_double]
        lib.pc_server_error.argtypes = [vp, ctypes.c_uint64]
        lib.pc_server_error.restype = ctypes.c_char_p
        lib.pc_server_outputs.argtypes = [vp, ctypes.c_uint64, vp, vp, vp]
        lib.pc_server_release.argtypes = [vp, ctypes.c_uint64]
        lib.pc_server_stats.argtypes = [vp, i64p, i64p]
        lib.pc_server_destroy.argtypes = [vp]
        lib.pc_extract_noalloc.argtypes = [ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, vp, vp, vp,
                                           ctypes.c_int64, ctypes.c_int64, i64p, i64p, vp]
        lib.pc_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        lib.pc_cell_counts.argtypes = [vp, i64p, ctypes.c_int, i64p]
        lib.pc_build_poset.argtypes = [vp]
        lib.pc_poset_level.argtypes = [vp, ctypes.c_int, i64p, i64p, vp, vp, vp]
        lib.pc_extract_domain.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp, ctypes.c_int64, vp,
                                          ctypes.c_int64, vp, vp]
        lib.pc_check_domain.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int64, vp, ctypes.c_int64, vp]
        lib.pc_last_error.argtypes = [vp]
        lib.pc_last_error.restype = ctypes.c_char_p
        for f in EXPORTS:
            if f not in ("pc_default_options", "pc_last_error", "pc_estimate_bytes", "pc_server_default_options",
                         "pc_server_error"):
                getattr(lib, f).restype = ctypes.c_int
        _libs[path] = lib
        return lib


def _addr(x) -> Optional[int]:
    """Address of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def _domain_arrays(dom):
    A = np.ascontiguousarray(dom.A, np.float64)
    c = np.ascontiguousarray(dom.c, np.float64)
    X0 = np.ascontiguousarray(dom.X0, np.float64)
    E0 = np.ascontiguousarray(dom.E0, np.int32)
    if A.ndim != 2 or c.shape != (A.shape[0],) or X0.ndim != 2 or X0.shape[1] != A.shape[1] or \
            E0.ndim != 2 or E0.shape[1] != 2:
        raise ValueError("domain arrays: A (m, D), c (m,), X0 (nv0, D), E0 (ne0, 2)")
    return A, c, X0, E0


def check_domain(dom) -> bool:
    """pc_check_domain: whether pc_extract_domain accepts the domain and its
    skeleton (host-only checks, no GPU needed)."""
    A, c, X0, E0 = _domain_arrays(dom)
    lib = load_library()
    return lib.pc_check_domain(A.shape[1], A.shape[0], _addr(A), _addr(c), X0.shape[0], _addr(X0), E0.shape[0],
                               _addr(E0)) == PC_OK


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


class Extractor:
    """One libpc context: extract complexes of ReLU MLPs on a box.

    precision: "fp32" | "mixed" (FP32 bulk, FP64 re-evaluation of signs within
    the FP32 error bound) | "fp64".  execution: "persistent" (one cooperative
    kernel per layer) | "stepwise" (one kernel per step and neuron).
    max_dim: the largest input dimension the context takes, 8 (libpc.so) or
    10 (libpc_d10.so, the same kernels with larger per-vertex arrays).
    debug_barrier_timeout: testing only; the persistent kernel's grid barriers
    time out on purpose (bounded), so extract() raises PC_ERR_TIMEOUT.
    kappa_audit: mixed precision; also checks (in FP64, without changing the
    result) the signs between kappa and kappa_audit error estimates, and
    counts those the filter let through wrong (diagnostics "missed").
    """

    def __init__(self, device: int = 0, precision: str = "mixed", execution: str = "persistent",
                 keep_tape: bool = False, strict: bool = False, init_vcap: int = 0, init_ecap: int = 0,
                 mem_budget_bytes: int = 0, kappa: float = 12.0, polish: int = -1, polish_tol: float = 1e-6,
                 timers: bool = False, torch_allocator: bool = True, gemm: str = "tensor",
                 pairing: str = "deferred", canonical: bool = False, prune: bool = False, max_dim: int = 8,
                 debug_barrier_timeout: bool = False, kappa_audit: float = 0.0):
        if not 1 <= max_dim <= 10:
            raise ValueError("max_dim must be in [1, 10]")
        self._lib = load_library(LIB if max_dim <= 8 else LIB_D10)
        o = Options()
        self._lib.pc_default_options(ctypes.byref(o))
        o.precision = PRECISION[precision]
        o.exec = EXEC[execution]
        o.keep_tape = int(keep_tape)
        o.strict = int(strict)
        o.init_vcap, o.init_ecap = int(init_vcap), int(init_ecap)
        o.mem_budget_bytes = int(mem_budget_bytes)
        o.filter_kappa = float(kappa)
        o.polish = int(polish)
        o.polish_tol = float(polish_tol)
        o.timers = int(timers)
        o.gemm = GEMM[gemm]
        o.pairing = PAIRING[pairing]
        o.canonical = int(canonical)
        o.prune = int(prune)
        o.debug_barrier_timeout = int(debug_barrier_timeout)
        o.filter_kappa_audit = float(kappa_audit)
        self.device = device
        self.options = o
        self._ctx = ctypes.c_void_p()
        self._check(self._lib.pc_create(ctypes.byref(self._ctx), device, ctypes.byref(o)))
        self._cb = None
        if torch_allocator:
            import torch

            def _alloc(size, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), device, int(stream or 0))
                except Exception:
                    return None

            def _free(ptr, size, stream, user):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            self._check(self._lib.pc_set_allocator(self._ctx, self._cb[0], self._cb[1], None))
        self.net = None

    def _check(self, st: int):
        if st != PC_OK:
            msg = self._lib.pc_last_error(self._ctx).decode() if getattr(self, "_ctx", None) else ""
            raise PcError(st, msg)

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.pc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- extraction -----------------------------------------------------------
    def extract(self, net, box, params=None, stream=None) -> "Extractor":
        """Runs pc_extract.  params: optional flat float64 parameters already
        on the device (torch tensor); else net.flat_params() from the host."""
        widths = np.ascontiguousarray(net.widths, np.int32)
        if params is None:
            params = np.ascontiguousarray(net.flat_params(), np.float64)
        lo = np.ascontiguousarray(box.lo, np.float64)
        hi = np.ascontiguousarray(box.hi, np.float64)
        self._keep = (widths, params, lo, hi)
        self.net = net
        st = self._lib.pc_extract(self._ctx, len(net.widths) - 1, _addr(widths), _addr(params),
                                  _addr(lo), _addr(hi), _stream_handle(stream))
        self._check(st)
        return self

    def extract_domain(self, net, dom, params=None, stream=None) -> "Extractor":
        """Runs pc_extract_domain on the polyhedral domain ``dom`` (A, c, X0,
        E0: {x : c - A x >= 0} and its 1-skeleton, e.g. workloads.Polytope)."""
        widths = np.ascontiguousarray(net.widths, np.int32)
        if params is None:
            params = np.ascontiguousarray(net.flat_params(), np.float64)
        arrs = _domain_arrays(dom)
        self._keep = (widths, params) + arrs
        self.net = net
        A, c, X0, E0 = arrs
        st = self._lib.pc_extract_domain(self._ctx, len(net.widths) - 1, _addr(widths), _addr(params), A.shape[0],
                                         _addr(A), _addr(c), X0.shape[0], _addr(X0), E0.shape[0], _addr(E0),
                                         _stream_handle(stream))
        self._check(st)
        return self

    def counts(self) -> dict:
        nv, ne = ctypes.c_int64(), ctypes.c_int64()
        sw, dim, nent = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.pc_counts(self._ctx, ctypes.byref(nv), ctypes.byref(ne), ctypes.byref(sw),
                                        ctypes.byref(dim), ctypes.byref(nent)))
        return {"nV": nv.value, "nE": ne.value, "S": sw.value, "D": dim.value, "P": nent.value}

    def vertices(self) -> np.ndarray:
        """(nV, D) float64 host copy."""
        c = self.counts()
        out = np.empty((c["D"], c["nV"]), np.float64)
        self._check(self._lib.pc_vertices(self._ctx, None, None, _addr(out)))
        return out.T

    def edges(self) -> np.ndarray:
        """(nE, 2) int32 host copy."""
        c = self.counts()
        out = np.empty((2, c["nE"]), np.int32)
        self._check(self._lib.pc_edges(self._ctx, None, None, _addr(out)))
        return np.ascontiguousarray(out.T)

    def sign_words(self) -> np.ndarray:
        """(S, nV) uint64 packed sign vectors, host copy."""
        c = self.counts()
        out = np.empty((c["S"], c["nV"]), np.uint64)
        self._check(self._lib.pc_signvectors(self._ctx, None, None, _addr(out)))
        return out

    def stats(self) -> np.ndarray:
        """(N, 8) int64: V before, E before, splits, keys, pairs, filtered, undecided, degenerate."""
        N = int(sum(self.net.widths[1:]))
        out = np.zeros((N, 8), np.int64)
        self._check(self._lib.pc_stats(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), N))
        return out

    def diagnostics(self) -> dict:
        out = np.zeros(15, np.int64)
        self._check(self._lib.pc_diagnostics(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 15))
        keys = ["launches", "grows", "polished", "degenerate", "undecided", "vcap", "ecap", "tcap",
                "bytes", "persistent_ctas", "reruns", "flips", "flip_margin_milli", "missed", "missed_margin_milli"]
        return dict(zip(keys, (int(x) for x in out)))

    def kernel_times_ms(self) -> np.ndarray:
        """(L, 2) ms per layer: forward product, neuron loop (-1: not measured)."""
        return self._times()[:-1].reshape(-1, 2)

    def polish_time_ms(self) -> float:
        return float(self._times()[-1])

    def _times(self) -> np.ndarray:
        L = len(self.net.widths) - 1
        out = np.full(2 * L + 1, -1.0)
        self._check(self._lib.pc_kernel_times(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              2 * L + 1))
        return out

    def values(self) -> np.ndarray:
        """(nV, H_L) last-layer pre-activations at the vertices (host copy)."""
        c = self.counts()
        H = self.net.widths[-1]
        dt = np.float64 if self.options.precision == PRECISION["fp64"] else np.float32
        out = np.empty((H, c["nV"]), dt)
        self._check(self._lib.pc_values(self._ctx, _addr(out)))
        return out.T

    def error_estimates(self):
        """(rho, coord_rms): per-vertex FP32 value scale and coordinate rms estimate."""
        n = self.counts()["nV"]
        rho = np.empty(n, np.float32)
        crd = np.empty(n, np.float32)
        self._check(self._lib.pc_error_estimates(self._ctx, _addr(rho), _addr(crd)))
        return rho, crd

    def device_arrays(self):
        """(X ptr, ld), (E ptr, ld), (SIG ptr, ld) of the context's device buffers."""
        res = []
        for f in (self._lib.pc_vertices, self._lib.pc_edges, self._lib.pc_signvectors):
            p, ld = ctypes.c_void_p(), ctypes.c_int64()
            self._check(f(self._ctx, ctypes.byref(p), ctypes.byref(ld), None))
            res.append((p.value, ld.value))
        return res

    def cell_counts(self):
        """(f_0, ..., f_D) k-cell counts of the last result and the Euler characteristic."""
        D = self.counts()["D"]
        f = np.zeros(D + 1, np.int64)
        chi = ctypes.c_int64()
        self._check(self._lib.pc_cell_counts(self._ctx, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), D + 1,
                                             ctypes.byref(chi)))
        return f, int(chi.value)

    def poset(self):
        """pc_build_poset then pc_poset_level for every level: a list over k
        = 0..D of (cells (n_k, S) uint64 packed sign words, row_ptr, parents),
        the CSR of the level-(k+1) cells containing each k-cell (None for k = D)."""
        self._check(self._lib.pc_build_poset(self._ctx))
        D, S = self.counts()["D"], self.counts()["S"]
        out = []
        for k in range(D + 1):
            n, nnz = ctypes.c_int64(), ctypes.c_int64()
            self._check(self._lib.pc_poset_level(self._ctx, k, ctypes.byref(n), ctypes.byref(nnz), None, None, None))
            cells = np.empty((n.value, S), np.uint64)
            rp = np.empty(n.value + 1, np.int64) if k < D else None
            cols = np.empty(max(nnz.value, 1), np.int64) if k < D else None
            self._check(self._lib.pc_poset_level(self._ctx, k, None, None, _addr(cells), _addr(rp), _addr(cols)))
            out.append((cells, rp, cols[:nnz.value] if cols is not None else None))
        return out

    def vertices_into(self, out) -> None:
        """Copies the D x nV coordinate block into `out` (host or device memory)."""
        self._check(self._lib.pc_vertices(self._ctx, None, None, _addr(out)))

    def backward(self, grad_x, grad_params, stream=None) -> None:
        """pc_backward: grad_x (D, nV) float64, grad_params flat float64 (host or device)."""
        self._check(self._lib.pc_backward(self._ctx, _addr(grad_x), _addr(grad_params), _stream_handle(stream)))


class Server:
    """The request loop of pc_server_*: submit extraction requests at any time,
    poll or wait for their results (latencies on the server's clock)."""

    def __init__(self, device: int = 0, max_slots: int = 8, precision: str = "mixed", execution: str = "stepwise",
                 polish: int = 0, keep_outputs: bool = False, mem_budget_bytes: int = 160 << 30,
                 request_max_bytes: int = 64 << 30):
        self._lib = load_library()
        o = ServerOptions()
        self._lib.pc_server_default_options(ctypes.byref(o))
        o.max_slots, o.precision, o.exec = max_slots, PRECISION[precision], EXEC[execution]
        o.polish, o.keep_outputs = int(polish), int(keep_outputs)
        o.mem_budget_bytes, o.request_max_bytes = int(mem_budget_bytes), int(request_max_bytes)
        self._s = ctypes.c_void_p()
        st = self._lib.pc_server_create(ctypes.byref(self._s), device, ctypes.byref(o))
        if st != PC_OK:
            raise PcError(st, "pc_server_create failed")
        self._nets = {}

    def submit(self, net, box) -> int:
        widths = np.ascontiguousarray(net.widths, np.int32)
        params = np.ascontiguousarray(net.flat_params(), np.float64)
        lo = np.ascontiguousarray(box.lo, np.float64)
        hi = np.ascontiguousarray(box.hi, np.float64)
        rid = ctypes.c_uint64()
        st = self._lib.pc_server_submit(self._s, len(net.widths) - 1, _addr(widths), _addr(params), _addr(lo),
                                        _addr(hi), ctypes.byref(rid))
        if st != PC_OK:
            raise PcError(st, "pc_server_submit failed")
        self._nets[rid.value] = net
        return rid.value

    def poll(self, rid: int):
        r = Result()
        st = self._lib.pc_server_poll(self._s, rid, ctypes.byref(r))
        return st, r

    def error(self, rid: int) -> str:
        return self._lib.pc_server_error(self._s, rid).decode()

    def wait_all(self, timeout_s: float = 600.0):
        st = self._lib.pc_server_wait_all(self._s, float(timeout_s))
        if st != PC_OK:
            raise PcError(st, "requests still pending")

    def outputs(self, rid: int):
        """(X (nV, D), S (S, nV) uint64, E (nE, 2)) of a finished request (keep_outputs)."""
        st, r = self.poll(rid)
        net = self._nets[rid]
        D = net.D
        S = (2 * D + net.n_neurons + 31) // 32
        X = np.empty((D, r.n_vertices), np.float64)
        E = np.empty((2, r.n_edges), np.int32)
        SIG = np.empty((S, r.n_vertices), np.uint64)
        st = self._lib.pc_server_outputs(self._s, rid, _addr(X), _addr(E), _addr(SIG))
        if st != PC_OK:
            raise PcError(st, "no outputs for this request")
        return X.T, SIG, np.ascontiguousarray(E.T)

    def stats(self):
        peak, cur = ctypes.c_int64(), ctypes.c_int64()
        self._lib.pc_server_stats(self._s, ctypes.byref(peak), ctypes.byref(cur))
        return {"peak_bytes": peak.value, "in_use_bytes": cur.value}

    def close(self):
        if getattr(self, "_s", None) and self._s.value:
            self._lib.pc_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_bytes(net) -> int:
    w = np.ascontiguousarray(net.widths, np.int32)
    return int(load_library().pc_estimate_bytes(len(net.widths) - 1, _addr(w)))
