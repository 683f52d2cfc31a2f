"""torch.autograd.Function over pc_extract / pc_backward.

Vertex coordinates as a differentiable function of the flat network
parameters (W1, b1, W2, b2, ...): the forward pass runs the CUDA extraction
(with the interpolation tape), the backward pass runs the CUDA adjoint
(pc_backward).  The complex's combinatorics are piecewise constant in the
parameters, so the gradient is that of the vertex positions with the
combinatorics held fixed.
"""
from __future__ import annotations

import torch


class ExtractVertices(torch.autograd.Function):
    """X = ExtractVertices.apply(params, extractor, net, box) -> (nV, D) float64.

    params: flat float64 CUDA tensor; extractor: an Extractor created with
    keep_tape=True (it keeps the sign vectors and edges of this extraction);
    net: a workloads.Net giving the widths; box: a workloads.Box.
    """

    @staticmethod
    def forward(ctx, params, extractor, net, box):
        p = params.detach().to(torch.float64).contiguous()
        extractor.extract(net, box, params=p)
        c = extractor.counts()
        X = torch.empty((c["D"], c["nV"]), dtype=torch.float64, device=params.device)
        extractor.vertices_into(X)
        ctx.extractor = extractor
        ctx.nparams = p.numel()
        return X.t()

    @staticmethod
    def backward(ctx, gX):
        g = gX.t().to(torch.float64).contiguous()
        out = torch.empty(ctx.nparams, dtype=torch.float64, device=g.device)
        ctx.extractor.backward(g, out)
        return out, None, None, None


def extract_vertices(params, extractor, net, box):
    return ExtractVertices.apply(params, extractor, net, box)
