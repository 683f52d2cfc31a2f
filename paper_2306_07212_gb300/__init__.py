"""GB300-native polyhedral-complex extraction from ReLU networks by edge subdivision.

The compute path is the CUDA library ``libpc.so`` (C ABI in ``include/pc.h``);
this package holds its thin ctypes binding, the build script and the seeded
workload generators.

Typical use::

    from paper_2306_07212_gb300 import Extractor, workloads
    net, box = workloads.torus_d3()
    with Extractor(precision="mixed") as ex:    # or "fp64", "fp32"
        ex.extract(net, box)                   # blocks until the result is ready
        X, E = ex.vertices(), ex.edges()       # (nV, D) float64, (nE, 2) int32
        S = ex.sign_words()                    # (S, nV) packed 2-bit sign vectors
        f, chi = ex.cell_counts()              # k-face counts, Euler characteristic

Options of ``Extractor``: ``execution`` ("persistent" | "stepwise"),
``canonical`` (fixed output order), ``prune`` (level-set extraction),
``keep_tape`` (for ``backward`` / ``autograd.extract_vertices``), ``gemm``
("tensor" | "simt" | "tensor3x"), ``pairing`` ("deferred" | "inline"),
``max_dim`` (8, or 10 for the build that takes D = 9, 10).
``Extractor.extract_domain`` takes a polyhedral domain (``workloads.Polytope``)
instead of a box; ``binding.Server`` serves many requests concurrently on
one GPU.
"""
from .binding import Extractor, PcError, load_library  # noqa: F401
from . import workloads  # noqa: F401
