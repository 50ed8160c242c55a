"""The strong split of perm(S_n) over GPUs (perm_schur_shard, sharding.py),
run here with every shard in one process on one GPU: the shards' partials
equal the oracle's Nijenhuis-Wilf range sums bit for bit, and the combined
integer equals the oracle's exact perm(S_n)."""
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def px():
    import torch
    assert torch.cuda.is_available()
    import paper_2602_10141_b300 as px
    return px


def test_shard_partials_match_oracle_range_sums(px):
    from paper_2602_10141_b300.sharding import shard_items, shard_range
    n, slices, world = 13, 3, 2
    k = px.perm_schur_prime_count(n)
    primes = px.perm_primes_1_mod_n(n, k + 1)
    for shard in range(world):
        got = px.perm_schur_shard(n, primes, slices, shard, world)
        want = [0] * len(primes)
        for i, j in shard_items(len(primes), slices, shard, world):
            p = primes[i]
            A = O.schur_residue_matrix(n, p, O.primitive_nth_root(p, n))
            k0, k1 = shard_range(n, slices, j)
            want[i] = (want[i] + O.ryser_nw_modp_gray_range(A, p, k0, k1)) % p
        assert got == want, shard


@pytest.mark.parametrize("n,slices,world", [(27, 4, 3), (31, 1, 8), (29, 5, 2)])
def test_all_shards_combine_to_the_oracle_integer(px, n, slices, world):
    """Shards summed mod p and combined by CRT give tests/golden/schur_crt_oracle.txt's
    perm(S_n) (written from the oracle alone) and perm_schur_crt's value."""
    from conftest import read_golden
    from paper_2602_10141_b300.sharding import combine
    want = {int(r[0]): int(r[1]) for r in read_golden("schur_crt_oracle.txt")}[n]
    k = px.perm_schur_prime_count(n)
    primes = px.perm_primes_1_mod_n(n, k + 1)
    sums = [0] * len(primes)
    for shard in range(world):
        for i, v in enumerate(px.perm_schur_shard(n, primes, slices, shard, world)):
            sums[i] = (sums[i] + v) % primes[i]
    value, residues = combine(n, primes, sums)
    assert value == want
    assert residues[:-1] == [want % p for p in primes[:-1]]


def test_shard_argument_errors(px):
    primes = px.perm_primes_1_mod_n(13, 2)
    for args in ((13, primes, 0, 0, 1), (13, primes, 2, 2, 2), (13, primes, 2, -1, 2), (0, primes, 1, 0, 1),
                 (13, [7], 1, 0, 1)):
        with pytest.raises(px.PermxError) as e:
            px.perm_schur_shard(*args)
        assert e.value.code == px.PERMX_EINVAL
