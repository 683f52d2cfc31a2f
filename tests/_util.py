"""Test helpers: canonical forms and independent numpy checks.

Nothing here implements the extraction.  The helpers put two results in the
same order (vertices sorted by sign vector, edges as sorted pairs of vertex
ranks) so they can be compared as sets, and evaluate networks with plain numpy
for the residual and direct-solve checks.
"""
from __future__ import annotations

import numpy as np


def unpack_codes(words: np.ndarray, P: int) -> np.ndarray:
    """Packed 2-bit codes (S, nV) uint64, word-major -> int8 (nV, P) in {-1,0,+1}.

    Entry j sits at bits 2*(j % 32) of word j // 32; 00 = 0, 01 = +, 10 = -.
    """
    words = np.asarray(words, dtype=np.uint64)
    nV = words.shape[1]
    out = np.zeros((nV, P), np.int8)
    for j in range(P):
        c = (words[j // 32] >> np.uint64(2 * (j % 32))) & np.uint64(3)
        out[:, j] = np.where(c == 1, 1, np.where(c == 2, -1, 0)).astype(np.int8)
        if np.any(c == 3):
            raise AssertionError(f"invalid code 11 at entry {j}")
    return out


def canon(X, S, E):
    """Sort vertices by sign vector; edges become sorted rank pairs, sorted."""
    S = np.asarray(S, np.int8)
    order = np.lexsort(S.T[::-1]) if S.shape[0] else np.zeros(0, np.int64)
    rank = np.empty(len(order), np.int64)
    rank[order] = np.arange(len(order))
    Ec = np.sort(rank[np.asarray(E, np.int64)], axis=1) if len(E) else np.zeros((0, 2), np.int64)
    if len(Ec):
        Ec = Ec[np.lexsort((Ec[:, 1], Ec[:, 0]))]
    return np.asarray(X)[order], S[order], Ec


def assert_same_complex(a, b, coord_tol=1e-9, what=""):
    """a, b: (X, S, E) triples. Sign vectors and edges bit-exact, X within tol."""
    Xa, Sa, Ea = canon(*a)
    Xb, Sb, Eb = canon(*b)
    assert Sa.shape == Sb.shape, f"{what}: vertex count / sign length {Sa.shape} vs {Sb.shape}"
    if not np.array_equal(Sa, Sb):
        diff = np.nonzero(np.any(Sa != Sb, axis=1))[0]
        raise AssertionError(f"{what}: {len(diff)} sign vectors differ (first rank {diff[:5]})")
    assert Ea.shape == Eb.shape, f"{what}: edge count {len(Ea)} vs {len(Eb)}"
    assert np.array_equal(Ea, Eb), f"{what}: edge sets differ"
    if len(Xa):
        err = np.max(np.abs(Xa - Xb))
        assert err <= coord_tol, f"{what}: max coordinate difference {err:.3e} > {coord_tol:.1e}"


def forward_all(net, X):
    """All pre-activations (nV, N) of a real forward pass, ReLU = max(0, z)."""
    a = np.asarray(X, np.float64)
    outs = []
    for W, b in zip(net.W, net.b):
        z = a @ W.T + b
        outs.append(z)
        a = np.maximum(z, 0.0)
    return np.concatenate(outs, axis=1)


def entry_values(net, box, X):
    """Values of every sign-vector entry (facets first) at points X, (nV, m+N)."""
    X = np.asarray(X, np.float64)
    D = X.shape[1]
    fac = np.empty((X.shape[0], 2 * D))
    fac[:, 0::2] = X - box.lo
    fac[:, 1::2] = box.hi - X
    return np.concatenate([fac, forward_all(net, X)], axis=1)


def affine_pieces(net, s):
    """Affine maps (G, c) of every entry under activation pattern from sign vector s."""
    D = net.D
    m = 2 * D
    G = np.zeros((m + net.n_neurons, D))
    c = np.zeros(m + net.n_neurons)
    for d in range(D):
        G[2 * d, d], c[2 * d] = 1.0, 0.0
        G[2 * d + 1, d], c[2 * d + 1] = -1.0, 0.0
    aG, ac = np.eye(D), np.zeros(D)
    off = m
    for W, b in zip(net.W, net.b):
        zG, zc = W @ aG, W @ ac + b
        H = W.shape[0]
        G[off:off + H], c[off:off + H] = zG, zc
        act = (s[off:off + H] == 1).astype(np.float64)
        aG, ac = zG * act[:, None], zc * act
        off += H
    return G, c


def solve_vertex(net, box, s):
    """Direct D x D solve of a vertex's zero entries on its own affine piece."""
    G, c = affine_pieces(net, s)
    D = net.D
    c = c.copy()
    c[0:2 * D:2] -= box.lo
    c[1:2 * D:2] += box.hi
    zs = np.nonzero(s == 0)[0]
    assert len(zs) == D, f"vertex has {len(zs)} zeros, expected {D}"
    return np.linalg.solve(G[zs], -c[zs])
