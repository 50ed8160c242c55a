"""The N > 1 path of bench.py on CPU: two gloo ranks take disjoint prime sets
(rank_prime_skip), each reconstructs the Schur permanent by CRT from its own
residues (computed here by the oracle, as the GPU is not used), and the
ranks agree; the max-over-ranks timing reduction is exercised too."""
import os
import socket

import torch.multiprocessing as mp

N_TEST = 11   # small Schur matrix so the oracle residues take milliseconds


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    import paper_2602_10141_b300 as px
    skip = bench.rank_prime_skip(rank)
    primes = px.perm_primes_1_mod_n(N_TEST, 5, skip)
    assert O.crt_modulus_suffices(N_TEST, primes)
    res = [O.perm_modp(O.schur_residue_matrix(N_TEST, p, px.perm_primitive_root(p, N_TEST)), p) for p in primes]
    value = px.perm_crt(res, primes)
    got = [None] * world
    dist.all_gather_object(got, (primes, value))
    t = torch.tensor([0.1 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((got, float(t.item())))
    dist.destroy_process_group()


def test_two_ranks_disjoint_primes_agree():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (p0, v0), (p1, v1) = got
    assert not set(p0) & set(p1)
    import oracle as O
    assert v0 == v1 == O.schur_exact(N_TEST)
    assert abs(tmax - 0.2) < 1e-12


# ---------------------------------------------------------------------------
# strong split of one perm(S_n) over ranks (paper_2602_10141_b300.sharding)
# ---------------------------------------------------------------------------

def _oracle_shard(n, primes, slices, shard, nshards):
    """A shard's partials from the oracle's Nijenhuis-Wilf range sums (the GPU
    is not used): the same items and ranges as the library's shard call."""
    import oracle as O
    from paper_2602_10141_b300.sharding import shard_items, shard_range
    out = [0] * len(primes)
    for i, j in shard_items(len(primes), slices, shard, nshards):
        p = primes[i]
        k0, k1 = shard_range(n, slices, j)
        A = O.schur_residue_matrix(n, p, O.primitive_nth_root(p, n))
        out[i] = (out[i] + O.ryser_nw_modp_gray_range(A, p, k0, k1)) % p
    return out


def _strong_worker(rank, world, port, slices, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2602_10141_b300 as px
    from paper_2602_10141_b300.sharding import schur_strong
    k = px.perm_schur_prime_count(N_TEST)
    primes = px.perm_primes_1_mod_n(N_TEST, k + 1)
    value, residues = schur_strong(N_TEST, primes, slices, shard_fn=_oracle_shard)
    got = [None] * world
    dist.all_gather_object(got, (value, residues))
    if rank == 0:
        q.put(got)
    dist.destroy_process_group()


def _run_strong(world, slices):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strong_worker, args=(r, world, port, slices, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


def test_strong_split_two_ranks_more_ranges_than_ranks():
    """world 2, 3 ranges per prime: every rank holds part of every prime;
    the gathered sums give the exact perm(S_11) on both ranks."""
    import oracle as O
    got = _run_strong(2, 3)
    assert got[0] == got[1]
    assert got[0][0] == O.schur_exact(N_TEST)


def test_strong_split_three_ranks_one_range_per_prime():
    """world 3, one range per prime (the ranks split the primes): same integer."""
    import oracle as O
    got = _run_strong(3, 1)
    assert got[0] == got[1] == got[2]
    assert got[0][0] == O.schur_exact(N_TEST)


def test_shard_partition_covers_every_range_once():
    from paper_2602_10141_b300.sharding import shard_items, shard_range
    for count, slices, world in ((6, 1, 8), (6, 3, 4), (5, 7, 3), (1, 1, 1), (2, 5, 16)):
        seen = []
        for r in range(world):
            seen += shard_items(count, slices, r, world)
        assert sorted(seen) == [(i, j) for i in range(count) for j in range(slices)]
        loads = [len(shard_items(count, slices, r, world)) for r in range(world)]
        assert max(loads) - min(loads) <= 1
    for n, slices in ((11, 3), (12, 1), (9, 7), (5, 40)):
        ranges = [shard_range(n, slices, j) for j in range(slices)]
        assert ranges[0][0] == 0 and ranges[-1][1] == 1 << (n - 1)
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))


def test_combine_rejects_a_wrong_residue():
    """The check prime catches a shard whose sum is wrong."""
    import pytest
    import oracle as O
    import paper_2602_10141_b300 as px
    from paper_2602_10141_b300.sharding import combine
    k = px.perm_schur_prime_count(N_TEST)
    primes = px.perm_primes_1_mod_n(N_TEST, k + 1)
    sums = _oracle_shard(N_TEST, primes, 2, 0, 1)
    assert combine(N_TEST, primes, sums)[0] == O.schur_exact(N_TEST)
    bad = list(sums)
    bad[0] = (bad[0] + 1) % primes[0]
    with pytest.raises(ArithmeticError):
        combine(N_TEST, primes, bad)
