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


def _q_positive_r(Z: torch.Tensor) -> torch.Tensor:
    """Q of the QR factorisation Z = QR whose R has a positive diagonal (unique
    for nonsingular Z), by Gram-Schmidt over the columns with every projection
    applied twice (CGS2, orthogonal to working precision).  For Gaussian Z this
    Q is Haar distributed (Mezzadri's recipe: QR, then R's diagonal phases
    folded into Q); batched over the leading dimension with O(n) tensor
    operations, where a library QR runs one small factorisation at a time."""
    Q = torch.empty_like(Z)
    n = Z.shape[-1]
    for j in range(n):
        v = Z[:, :, j]
        if j:
            Qj = Q[:, :, :j]
            for _ in range(2):
                c = torch.einsum("bij,bi->bj", Qj.conj(), v)
                v = v - torch.einsum("bij,bj->bi", Qj, c)
        Q[:, :, j] = v / torch.linalg.vector_norm(v, dim=1, keepdim=True)
    return Q


def batch(name: str, n: int, count: int, seed: int, device="cuda") -> torch.Tensor:
    """(count, n, n) matrices of one ensemble, contiguous on the device."""
    g = _gen(seed, device)
    if name == "haar_u":
        return _q_positive_r(_cn(count, n, g, device)).contiguous()
    if name == "haar_o":
        Z = torch.randn((count, n, n), generator=g, device=device, dtype=torch.float64)
        return _q_positive_r(Z).contiguous()
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
