"""Seeded ensemble generation on the GPU for throughput runs (inputs only).

The same recipes as ``ensembles.py`` (paper §3.1, §5.1, §6), drawn with a
seeded ``torch.Generator`` on the device so that batches of tens of thousands
of matrices need no host round trip.  Every batch is reproducible from its
seed; a subsample can be copied back and checked against the oracle.
"""
from __future__ import annotations

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def _cn(count, n, g, device, var=1.0):
    s = (var / 2.0) ** 0.5
    re = torch.randn((count, n, n), generator=g, device=device, dtype=torch.float64) * s
    im = torch.randn((count, n, n), generator=g, device=device, dtype=torch.float64) * s
    return torch.complex(re, im)


def batch(name: str, n: int, count: int, seed: int, device="cuda") -> torch.Tensor:
    """(count, n, n) matrices of one ensemble, contiguous on the device."""
    g = _gen(seed, device)
    if name == "haar_u":
        Q, R = torch.linalg.qr(_cn(count, n, g, device))
        d = torch.diagonal(R, dim1=-2, dim2=-1)
        return (Q * (d / d.abs()).unsqueeze(-2)).contiguous()
    if name == "haar_o":
        Z = torch.randn((count, n, n), generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(Z)
        s = torch.sign(torch.diagonal(R, dim1=-2, dim2=-1))
        s[s == 0] = 1.0
        return (Q * s.unsqueeze(-2)).contiguous()
    if name == "gue":
        A = _cn(count, n, g, device)
        return ((A + A.conj().transpose(-1, -2)) / 2).contiguous()
    if name == "goe":
        A = torch.randn((count, n, n), generator=g, device=device, dtype=torch.float64)
        return ((A + A.transpose(-1, -2)) / 2).contiguous()
    if name == "ginibre_c":
        return _cn(count, n, g, device).contiguous()
    if name == "ginibre_r":
        return torch.randn((count, n, n), generator=g, device=device, dtype=torch.float64).contiguous()
    raise ValueError(name)
