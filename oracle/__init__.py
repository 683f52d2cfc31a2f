"""FP64 CPU oracle for edge subdivision (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does.  The C++ source in ``oracle.cpp`` is written
from the paper and shares no code with the CUDA path.

Functions
  extract(net, box, max_neurons=-1, prune=False)
                                     edge subdivision (Section 4.2); with
                                     prune, the pruning during subdivision of
                                     Section 5.4.2 (level-set extraction)
  brute(net, box, tol)               the complex from its definition
  extract_domain(net, dom), brute_domain(net, dom)
                                     the same on a polyhedral domain of
                                     half-spaces (e.g. a simplex)
  faces(result)                      k-cell counts by perturbation (Section 4.1)
  grad(net, result, gx)              implicit-function gradient of a vertex loss
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain -O2, portable)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32p, f64p, i64p = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64))
            lib.orc_extract.restype = vp
            lib.orc_extract.argtypes = [ctypes.c_int, i32p, f64p, f64p, f64p, ctypes.c_int, ctypes.c_int]
            lib.orc_layer_counts.argtypes = [vp, i64p]
            lib.orc_extract_domain.restype = vp
            lib.orc_extract_domain.argtypes = [ctypes.c_int, i32p, f64p, ctypes.c_int, f64p, f64p, ctypes.c_int64,
                                               f64p, ctypes.c_int64, i32p, ctypes.c_int, ctypes.c_int]
            lib.orc_brute_domain.restype = vp
            lib.orc_brute_domain.argtypes = [ctypes.c_int, i32p, f64p, ctypes.c_int, f64p, f64p, ctypes.c_double]
            lib.orc_brute.restype = vp
            lib.orc_brute.argtypes = [ctypes.c_int, i32p, f64p, f64p, f64p, ctypes.c_double]
            lib.orc_free.argtypes = [vp]
            lib.orc_status.argtypes = [vp]
            lib.orc_error.restype = ctypes.c_char_p
            lib.orc_error.argtypes = [vp]
            for f in (lib.orc_nv, lib.orc_ne):
                f.restype = ctypes.c_int64
                f.argtypes = [vp]
            lib.orc_nsig.argtypes = [vp]
            lib.orc_vertices.argtypes = [vp, f64p]
            lib.orc_signs.argtypes = [vp, ctypes.POINTER(ctypes.c_int8)]
            lib.orc_edges.argtypes = [vp, i32p]
            lib.orc_stats.argtypes = [vp, i64p]
            lib.orc_faces.restype = ctypes.c_int64
            lib.orc_faces.argtypes = [vp, i64p]
            lib.orc_grad.argtypes = [vp, ctypes.c_int, i32p, f64p, f64p, f64p]
            lib.orc_poset.restype = vp
            lib.orc_poset.argtypes = [vp]
            lib.orc_poset_status.argtypes = [vp]
            lib.orc_poset_error.restype = ctypes.c_char_p
            lib.orc_poset_error.argtypes = [vp]
            for f in (lib.orc_poset_count, lib.orc_poset_nnz):
                f.restype = ctypes.c_int64
                f.argtypes = [vp, ctypes.c_int]
            lib.orc_poset_cells.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int8)]
            lib.orc_poset_incidence.argtypes = [vp, ctypes.c_int, i64p, i64p]
            lib.orc_poset_free.argtypes = [vp]
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclasses.dataclass
class Result:
    """One extracted complex: vertices X (nV, D), sign vectors S (nV, m+N) in
    {-1,0,+1}, edges E (nE, 2), per-neuron stats (N, 4) = nsplit, nkeys,
    npairs, ndegenerate, and a status (0 ok, 4 degenerate, 5 pairing)."""

    X: np.ndarray
    S: np.ndarray
    E: np.ndarray
    stats: np.ndarray
    status: int
    error: str
    D: int
    _handle: object = None

    @property
    def nV(self):
        return self.X.shape[0]

    @property
    def nE(self):
        return self.E.shape[0]


def _collect(lib, h, D, with_stats=True, m=None):
    nV, nE, P = lib.orc_nv(h), lib.orc_ne(h), lib.orc_nsig(h)
    X = np.empty((nV, D), np.float64)
    S = np.empty((nV, P), np.int8)
    E = np.empty((nE, 2), np.int32)
    if nV:
        lib.orc_vertices(h, _ptr(X, ctypes.c_double))
        lib.orc_signs(h, _ptr(S, ctypes.c_int8))
    if nE:
        lib.orc_edges(h, _ptr(E, ctypes.c_int32))
    N = P - (2 * D if m is None else m)
    stats = np.zeros((N, 4), np.int64)
    if with_stats and N:
        lib.orc_stats(h, _ptr(stats, ctypes.c_int64))
    return X, S, E, stats


def _net_args(net, box):
    widths = np.ascontiguousarray(net.widths, np.int32)
    params = np.ascontiguousarray(net.flat_params(), np.float64)
    lo = np.ascontiguousarray(box.lo, np.float64)
    hi = np.ascontiguousarray(box.hi, np.float64)
    return widths, params, lo, hi


class _Handle:
    def __init__(self, lib, h):
        self.lib, self.h = lib, h

    def __del__(self):
        try:
            self.lib.orc_free(self.h)
        except Exception:
            pass


def extract(net, box, max_neurons: int = -1, prune: bool = False) -> Result:
    lib = _load()
    widths, params, lo, hi = _net_args(net, box)
    h = lib.orc_extract(net.L, _ptr(widths, ctypes.c_int32), _ptr(params, ctypes.c_double),
                        _ptr(lo, ctypes.c_double), _ptr(hi, ctypes.c_double), int(max_neurons), int(prune))
    X, S, E, stats = _collect(lib, h, net.D)
    return Result(X, S, E, stats, lib.orc_status(h), lib.orc_error(h).decode(), net.D, _Handle(lib, h))


def _domain_args(dom):
    A = np.ascontiguousarray(dom.A, np.float64)
    c = np.ascontiguousarray(dom.c, np.float64)
    X0 = np.ascontiguousarray(dom.X0, np.float64)
    E0 = np.ascontiguousarray(dom.E0, np.int32)
    return A, c, X0, E0


def extract_domain(net, dom, max_neurons: int = -1, prune: bool = False) -> Result:
    """Edge subdivision on a polyhedral domain (half-spaces dom.c - dom.A x >= 0,
    initial skeleton dom.X0, dom.E0)."""
    lib = _load()
    widths, params, _, _ = _net_args(net, type("B", (), {"lo": np.zeros(1), "hi": np.zeros(1)}))
    A, c, X0, E0 = _domain_args(dom)
    h = lib.orc_extract_domain(net.L, _ptr(widths, ctypes.c_int32), _ptr(params, ctypes.c_double), len(c),
                               _ptr(A, ctypes.c_double), _ptr(c, ctypes.c_double), len(X0),
                               _ptr(X0, ctypes.c_double), len(E0), _ptr(E0, ctypes.c_int32), int(max_neurons),
                               int(prune))
    X, S, E, stats = _collect(lib, h, net.D, m=len(c))
    return Result(X, S, E, stats, lib.orc_status(h), lib.orc_error(h).decode(), net.D, _Handle(lib, h))


def brute_domain(net, dom, tol: float = 1e-9) -> Result:
    """The complex from its definition on a polyhedral domain."""
    lib = _load()
    widths, params, _, _ = _net_args(net, type("B", (), {"lo": np.zeros(1), "hi": np.zeros(1)}))
    A, c, _, _ = _domain_args(dom)
    h = lib.orc_brute_domain(net.L, _ptr(widths, ctypes.c_int32), _ptr(params, ctypes.c_double), len(c),
                             _ptr(A, ctypes.c_double), _ptr(c, ctypes.c_double), float(tol))
    X, S, E, _ = _collect(lib, h, net.D, with_stats=False, m=len(c))
    return Result(X, S, E, np.zeros((0, 4), np.int64), lib.orc_status(h), lib.orc_error(h).decode(), net.D,
                  _Handle(lib, h))


def layer_counts(res: Result) -> np.ndarray:
    """(layers, 2) vertices and edges after each completed layer (and its pruning)."""
    lib = _load()
    out = np.zeros((64, 2), np.int64)
    n = lib.orc_layer_counts(res._handle.h, _ptr(out, ctypes.c_int64))
    return out[:n]


def brute(net, box, tol: float = 1e-9) -> Result:
    lib = _load()
    widths, params, lo, hi = _net_args(net, box)
    h = lib.orc_brute(net.L, _ptr(widths, ctypes.c_int32), _ptr(params, ctypes.c_double),
                      _ptr(lo, ctypes.c_double), _ptr(hi, ctypes.c_double), float(tol))
    X, S, E, _ = _collect(lib, h, net.D, with_stats=False)
    return Result(X, S, E, np.zeros((0, 4), np.int64), lib.orc_status(h),
                  lib.orc_error(h).decode(), net.D, _Handle(lib, h))


def faces(res: Result):
    """(f_0, ..., f_D) cell counts by perturbation and the Euler characteristic."""
    lib = _load()
    f = np.zeros(res.D + 1, np.int64)
    chi = lib.orc_faces(res._handle.h, _ptr(f, ctypes.c_int64))
    return f, int(chi)


@dataclasses.dataclass
class Poset:
    """The face poset of an extracted complex (Section 4.1).  cells[k]: the
    k-cells' sign vectors (n_k, m+N) int8, sorted lexicographically (-1 < 0
    < +1); parents[k] (k < D): CSR (row_ptr (n_k + 1,), cols) of the
    (k+1)-cells containing each k-cell, its zeros perturbed in entry order,
    + before -.  status 0, or 5 when a perturbed vertex is not an edge."""

    cells: list
    parents: list
    status: int
    error: str


def poset(res: Result) -> Poset:
    lib = _load()
    q = lib.orc_poset(res._handle.h)
    try:
        P = res.S.shape[1]
        cells, parents = [], []
        for k in range(res.D + 1):
            n = lib.orc_poset_count(q, k)
            c = np.empty((n, P), np.int8)
            if n:
                lib.orc_poset_cells(q, k, _ptr(c, ctypes.c_int8))
            cells.append(c)
            if k < res.D:
                nnz = lib.orc_poset_nnz(q, k)
                rp = np.empty(n + 1, np.int64)
                cl = np.empty(max(nnz, 1), np.int64)
                lib.orc_poset_incidence(q, k, _ptr(rp, ctypes.c_int64), _ptr(cl, ctypes.c_int64))
                parents.append((rp, cl[:nnz]))
        return Poset(cells, parents, lib.orc_poset_status(q), lib.orc_poset_error(q).decode())
    finally:
        lib.orc_poset_free(q)


def grad(net, res: Result, gx: np.ndarray) -> np.ndarray:
    """dL/dtheta (flat W1,b1,W2,b2,... layout) for vertex-position gradients gx (nV, D)."""
    lib = _load()
    widths, params, _, _ = _net_args(net, type("B", (), {"lo": np.zeros(1), "hi": np.zeros(1)}))
    gx = np.ascontiguousarray(gx, np.float64)
    assert gx.shape == (res.nV, res.D)
    out = np.zeros(params.size, np.float64)
    rc = lib.orc_grad(res._handle.h, net.L, _ptr(widths, ctypes.c_int32), _ptr(params, ctypes.c_double),
                      _ptr(gx, ctypes.c_double), _ptr(out, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle gradient failed (status {rc})")
    return out
