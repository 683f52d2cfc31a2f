"""Seeded synthetic inputs: ReLU MLPs and box domains.

This module only *draws* networks, domains and request streams. It holds none
of the extraction arithmetic, so both the CUDA path and the FP64 oracle can take
their inputs from it without sharing any of the method.

Conventions (Section 3.4, Eq. 4): a network with widths ``[D, H_1, ..., H_L]``
has ``W[l]`` of shape ``(H_{l+1}, H_l)`` (out x in, so ``z = W x + b``) and
``b[l]`` of length ``H_{l+1}``.  Every layer's pre-activation zero set is a
folded hyperplane, the last (output) layer included.

Draw recipe: ``numpy.random.default_rng(seed)``; weights and biases are drawn in
the order W1, b1, W2, b2, ... as float64 standard normals scaled by
``sqrt(2 / fan_in)`` (He-normal) and ``sqrt(bias_var)`` respectively; a bias
variance of 0.01 gives a bias standard deviation of 0.1.  The counting sweep
draws both uniformly on [-1/sqrt(fan_in), 1/sqrt(fan_in)] instead.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import List, Optional, Sequence

import numpy as np

_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


@dataclasses.dataclass
class Net:
    """A ReLU MLP in float64; ``widths[0]`` is the input dimension D."""

    widths: List[int]
    W: List[np.ndarray]
    b: List[np.ndarray]

    @property
    def D(self) -> int:
        return int(self.widths[0])

    @property
    def L(self) -> int:
        return len(self.widths) - 1

    @property
    def n_neurons(self) -> int:
        return int(sum(self.widths[1:]))

    def flat_params(self) -> np.ndarray:
        """W1, b1, W2, b2, ... concatenated (row-major W)."""
        parts = []
        for W, b in zip(self.W, self.b):
            parts.append(np.ascontiguousarray(W, dtype=np.float64).ravel())
            parts.append(np.ascontiguousarray(b, dtype=np.float64).ravel())
        return np.concatenate(parts)

    def with_flat_params(self, theta: np.ndarray) -> "Net":
        theta = np.asarray(theta, dtype=np.float64)
        W, b, off = [], [], 0
        for l in range(self.L):
            o, i = self.widths[l + 1], self.widths[l]
            W.append(theta[off:off + o * i].reshape(o, i).copy())
            off += o * i
            b.append(theta[off:off + o].copy())
            off += o
        return Net(list(self.widths), W, b)

    def rounded_to_fp32(self) -> "Net":
        return Net(list(self.widths),
                   [w.astype(np.float32).astype(np.float64) for w in self.W],
                   [v.astype(np.float32).astype(np.float64) for v in self.b])


@dataclasses.dataclass
class Box:
    lo: np.ndarray
    hi: np.ndarray

    @staticmethod
    def cube(D: int, half: float = 1.0) -> "Box":
        return Box(np.full(D, -half), np.full(D, half))


def he_normal_mlp(widths: Sequence[int], seed: int, bias_var: float = 0.01) -> Net:
    """He-normal weights N(0, 2/fan_in) and biases N(0, bias_var), float64."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for l in range(len(widths) - 1):
        fan_in, fan_out = int(widths[l]), int(widths[l + 1])
        W.append(rng.standard_normal((fan_out, fan_in)) * math.sqrt(2.0 / fan_in))
        b.append(rng.standard_normal(fan_out) * math.sqrt(bias_var))
    return Net([int(w) for w in widths], W, b)


# --- the five workloads -----------------------------------------------------

def small_d2() -> tuple:
    """D=2, box [-1,1]^2, MLP 2-8-8-1, He-normal weights, biases N(0,0.01), seed 0."""
    return he_normal_mlp([2, 8, 8, 1], seed=0), Box.cube(2)


TORUS_FILE = os.path.join(_DATA, "torus_3x64x4x1.npz")


def torus_d3() -> tuple:
    """D=3 torus SDF net 3-64-64-64-64-1 (FP32 weights from a 2000-step Adam fit).

    The weights were produced once by ``data/make_torus_net.py`` and stored;
    they are exactly representable in float64.
    """
    with np.load(TORUS_FILE) as f:
        widths = [int(x) for x in f["widths"]]
        W = [f[f"W{l}"].astype(np.float64) for l in range(len(widths) - 1)]
        b = [f[f"b{l}"].astype(np.float64) for l in range(len(widths) - 1)]
    return Net(widths, W, b), Box.cube(3)


@dataclasses.dataclass
class Polytope:
    """A bounded domain {x : c - A x >= 0} with its 1-skeleton (vertices X0,
    edges E0 as index pairs)."""

    A: np.ndarray
    c: np.ndarray
    X0: np.ndarray
    E0: np.ndarray

    @property
    def D(self) -> int:
        return self.A.shape[1]

    @staticmethod
    def simplex(D: int, lo: float = -1.0, size: float = 2.0) -> "Polytope":
        """{x_d >= lo for all d, sum_d (x_d - lo) <= size}: D + 1 vertices
        (the corner lo and lo + size e_d), every pair an edge."""
        A = np.vstack([-np.eye(D), np.ones((1, D))])
        c = np.concatenate([np.full(D, -lo), [size + D * lo]])
        X0 = np.vstack([np.full(D, lo)] + [np.full(D, lo) + size * np.eye(D)[d] for d in range(D)])
        E0 = np.array([(i, j) for i in range(D + 1) for j in range(i + 1, D + 1)], np.int32)
        return Polytope(A, c, X0, E0)

    @staticmethod
    def corner_cut(D: int) -> "Polytope":
        """[-1,1]^D without the corner (1, ..., 1): the box's 2D half-spaces
        and sum_d x_d <= D - 1.  A simple polytope with the 2^D - 1 remaining
        corners and D new vertices (1, ..., 1 with one coordinate 0)."""
        box = Polytope.from_box(Box.cube(D))
        A = np.vstack([box.A, np.ones((1, D))])
        c = np.concatenate([box.c, [D - 1.0]])
        full = (1 << D) - 1
        keep = [k for k in range(1 << D) if k != full]
        rank = {k: r for r, k in enumerate(keep)}
        X0 = [box.X0[k] for k in keep]
        E0 = [(rank[u], rank[w]) for u, w in box.E0 if full not in (u, w)]
        for d in range(D):
            X0.append(np.where(np.arange(D) == d, 0.0, 1.0))
            E0.append((rank[full ^ (1 << d)], len(X0) - 1))  # the cut edge toward the removed corner
        first = len(keep)
        E0 += [(first + i, first + j) for i in range(D) for j in range(i + 1, D)]
        return Polytope(A, c, np.array(X0), np.array(E0, np.int32))

    @staticmethod
    def from_box(box: "Box") -> "Polytope":
        """The box as 2D half-spaces (2d: x_d - lo_d >= 0, 2d+1: hi_d - x_d >= 0)
        with its corners (corner c has coordinate d at hi iff bit d of c is set)
        and axis edges, in the order the box extraction uses."""
        D = len(box.lo)
        A = np.zeros((2 * D, D))
        c = np.zeros(2 * D)
        for d in range(D):
            A[2 * d, d], c[2 * d] = -1.0, -box.lo[d]
            A[2 * d + 1, d], c[2 * d + 1] = 1.0, box.hi[d]
        X0 = np.array([[box.hi[d] if (k >> d) & 1 else box.lo[d] for d in range(D)] for k in range(1 << D)])
        E0 = np.array([(k, k | (1 << d)) for d in range(D) for k in range(1 << D) if not (k >> d) & 1], np.int32)
        return Polytope(A, c, X0, E0)


def precision_d4(seed: int = 0) -> tuple:
    """D=4, box [-1,1]^4, MLP 4-128-128-128-1 He-normal, rounded once to FP32."""
    return he_normal_mlp([4, 128, 128, 128, 1], seed=seed).rounded_to_fp32(), Box.cube(4)


def precision_d4_subbox(half_width: float = 0.02, seed: int = 0) -> tuple:
    """The D=4 precision network on the centred sub-box [-h, h]^4.

    The full box holds far more cells than the oracle (or device memory) can
    take: the first layer alone can have up to C(128, 4) ~ 1e7 interior
    vertices.  h = 0.02 gives about 2e5 vertices and 8e5 edges.
    """
    net, _ = precision_d4(seed)
    return net, Box(np.full(4, -half_width), np.full(4, half_width))


def diff_d3(seed: int = 0) -> tuple:
    """D=3, box [-1,1]^3, MLP 3-32-32-32-1 He-normal, rounded to FP32."""
    return he_normal_mlp([3, 32, 32, 32, 1], seed=seed).rounded_to_fp32(), Box.cube(3)


def random_mlp(D: int, depth: int, width: int, seed: int) -> tuple:
    """A generic random net: ``depth`` hidden layers of ``width`` and one output."""
    widths = [D] + [width] * depth + [1]
    return he_normal_mlp(widths, seed=seed), Box.cube(D)


def default_uniform_mlp(widths: Sequence[int], seed: int) -> Net:
    """Weights and biases uniform on [-1/sqrt(fan_in), 1/sqrt(fan_in)], float64.

    This is the distribution of a freshly constructed fully-connected layer in
    PyTorch (Kaiming-uniform with a = sqrt(5) gives the same bound for W).
    Drawn in the order W1, b1, W2, b2, ... from ``default_rng(seed)``.
    """
    rng = np.random.default_rng(seed)
    W, b = [], []
    for l in range(len(widths) - 1):
        fan_in, fan_out = int(widths[l]), int(widths[l + 1])
        bound = 1.0 / math.sqrt(fan_in)
        W.append(rng.uniform(-bound, bound, (fan_out, fan_in)))
        b.append(rng.uniform(-bound, bound, fan_out))
    return Net([int(w) for w in widths], W, b)


COUNTING_DIMS = tuple(range(1, 11))
COUNTING_WIDTHS = (10, 20, 40)
COUNTING_SEEDS = 5


def counting_sweep_net(D: int, width: int, seed: int) -> tuple:
    """One point of the counting sweep of Section 5.1.2: a randomly initialised
    net of four hidden layers of ``width`` and a scalar output, on [-1,1]^D.

    The paper sweeps D = 1..10 and widths 10, 20, 40 with five random nets per
    point and reports vertex and edge counts, run time and peak device memory.
    The weights are drawn as a fresh PyTorch layer would draw them and rounded
    once to FP32, so every precision mode extracts the same net.
    """
    widths = [D] + [width] * 4 + [1]
    return default_uniform_mlp(widths, seed=seed).rounded_to_fp32(), Box.cube(D)


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    net: Net
    box: Box


def serving_stream(n_requests: int = 2000, rate_per_s: float = 200.0, seed: int = 0,
                   dims=(2, 3, 4), depths=(2, 3, 4, 5, 6),
                   widths=(16, 32, 64, 128)) -> List[Request]:
    """Poisson arrivals (exponential gaps, mean 1/rate) of random extraction requests.

    Request k draws D, depth and width from its own generator seeded with k,
    then He-normal weights (rounded to FP32) from seed k.
    """
    gaps = np.random.default_rng(seed).exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for k in range(n_requests):
        r = np.random.default_rng(1_000_003 + k)
        D = int(r.choice(dims))
        depth = int(r.choice(depths))
        width = int(r.choice(widths))
        net = he_normal_mlp([D] + [width] * depth + [1], seed=k).rounded_to_fp32()
        out.append(Request(k, float(t[k]), net, Box.cube(D)))
    return out


def torus_sdf(p: np.ndarray, R: float = 0.6, r: float = 0.25) -> np.ndarray:
    """Signed distance to a torus around the z axis (major radius R, minor r)."""
    q = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2) - R
    return np.sqrt(q ** 2 + p[:, 2] ** 2) - r
