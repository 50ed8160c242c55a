"""Strong split of exact perm(S_n) over several GPUs, one process per GPU
(paper §2.1: residues mod independent primes, recombined by CRT; §2.2: the
Gray-code blocks of one prime are independent too).

Every prime's Nijenhuis-Wilf walk of 2^(n-1) Gray indices is cut into
``slices`` equal ranges; work item w = i * slices + j (prime i, range j)
belongs to rank w mod world, so N ranks finish one problem about N times
faster whether they outnumber the primes or not.  Each rank computes the
signed sums of its ranges on its GPU (``perm_schur_shard`` in the C-ABI),
the ranks exchange one residue per prime (``all_gather``: the only data
collective), every rank adds them mod p, applies the walk's factor
2 (-1)^(n-1) and reconstructs the integer by CRT over all primes but the
last, which checks the result.
"""
from __future__ import annotations

from typing import Callable, Sequence

ShardFn = Callable[[int, Sequence[int], int, int, int], Sequence[int]]


def shard_items(count: int, slices: int, shard: int, nshards: int) -> list[tuple[int, int]]:
    """The (prime index, range index) items of one shard, in the order the
    library walks them (the same rule as perm_schur_shard)."""
    return [(i, j) for i in range(count) for j in range(slices) if (i * slices + j) % nshards == shard]


def shard_range(n: int, slices: int, j: int) -> tuple[int, int]:
    """Gray indices [k0, k1) of range j of the 2^(n-1)-index walk (possibly empty)."""
    total = 1 << (n - 1)
    length = -(-total // slices)
    return min(j * length, total), min((j + 1) * length, total)


def combine(n: int, primes: Sequence[int], partial_sums: Sequence[int]) -> tuple[int, list[int]]:
    """perm(S_n) from the ranks' summed partials (one per prime, already
    reduced mod that prime): residues r_i = 2 (-1)^(n-1) s_i mod p_i, CRT over
    primes[:-1], the last prime checks.  Returns (value, residues)."""
    import paper_2602_10141_b300 as px
    res = []
    for s, p in zip(partial_sums, primes):
        v = 2 * int(s) % p
        res.append((p - v) % p if (n - 1) % 2 else v)
    value = px.perm_crt(res[:-1], list(primes[:-1]))
    if value % primes[-1] != res[-1]:
        raise ArithmeticError("CRT check failed: the check prime's residue disagrees with the reconstruction")
    return value, res


def gpu_shard(n: int, primes: Sequence[int], slices: int, shard: int, nshards: int) -> list[int]:
    """This rank's partial sums on its current GPU (perm_schur_shard)."""
    import paper_2602_10141_b300 as px
    return px.perm_schur_shard(n, primes, slices, shard, nshards)


def schur_strong(n: int, primes: Sequence[int], slices: int, shard_fn: ShardFn | None = None) -> tuple[int, list[int]]:
    """perm(S_n) over the ranks of the default torch.distributed process group
    (or alone without one).  ``shard_fn`` computes one shard's partials
    (default: this rank's GPU).  Every rank returns (value, residues)."""
    import torch
    import torch.distributed as dist
    shard_fn = shard_fn or gpu_shard
    dist_on = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank() if dist_on else 0
    world = dist.get_world_size() if dist_on else 1
    part = [int(x) for x in shard_fn(n, primes, slices, rank, world)]
    if world > 1:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
        mine = torch.tensor(part, dtype=torch.int64, device=dev)
        got = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(got, mine)
        sums = [0] * len(primes)
        for t in got:
            for i, v in enumerate(t.cpu().tolist()):
                sums[i] = (sums[i] + int(v)) % primes[i]
    else:
        sums = part
    return combine(n, primes, sums)
