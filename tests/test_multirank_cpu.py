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
