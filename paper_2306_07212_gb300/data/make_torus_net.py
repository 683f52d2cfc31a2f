"""Fit the D=3 torus workload network and store its FP32 weights.

Recipe: 2^16 points uniform in [-1,1]^3 (torch generator, seed 0), target the
signed distance to a torus around the z axis (R=0.6, r=0.25); an MLP
3-64-64-64-64-1 with ReLU and PyTorch's default ``nn.Linear`` initialisation
under ``torch.manual_seed(0)``; full-batch mean-squared error, Adam with
lr 1e-3, 2000 steps, float32, single CPU thread (for repeatability).

Run once: ``python paper_2306_07212_gb300/data/make_torus_net.py``.
The output ``torus_3x64x4x1.npz`` is the input of the D=3 workload.
"""
import os
import sys

import numpy as np
import torch


def main(out=None, steps=2000):
    torch.set_num_threads(1)
    torch.manual_seed(0)
    g = torch.Generator().manual_seed(0)
    pts = torch.rand((1 << 16, 3), generator=g, dtype=torch.float32) * 2 - 1
    q = torch.sqrt(pts[:, 0] ** 2 + pts[:, 1] ** 2) - 0.6
    sdf = (torch.sqrt(q ** 2 + pts[:, 2] ** 2) - 0.25)[:, None]
    widths = [3, 64, 64, 64, 64, 1]
    layers = []
    for l in range(len(widths) - 1):
        layers.append(torch.nn.Linear(widths[l], widths[l + 1]))
        if l < len(widths) - 2:
            layers.append(torch.nn.ReLU())
    net = torch.nn.Sequential(*layers)
    opt = torch.optim.Adam(net.parameters(), lr=1e-3)
    for it in range(steps):
        opt.zero_grad()
        loss = torch.mean((net(pts) - sdf) ** 2)
        loss.backward()
        opt.step()
        if it % 500 == 0 or it == steps - 1:
            print(f"step {it} mse {loss.item():.3e}", file=sys.stderr)
    lin = [m for m in net if isinstance(m, torch.nn.Linear)]
    arrays = {"widths": np.array(widths, dtype=np.int32)}
    for l, m in enumerate(lin):
        arrays[f"W{l}"] = m.weight.detach().numpy().astype(np.float32)
        arrays[f"b{l}"] = m.bias.detach().numpy().astype(np.float32)
    out = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "torus_3x64x4x1.npz")
    np.savez(out, **arrays)
    print(f"wrote {out} final mse {loss.item():.3e}", file=sys.stderr)


if __name__ == "__main__":
    main()
