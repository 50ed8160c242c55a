"""Checkpoint files are validated on the host before any GPU work: a corrupt
file or one from a different run is rejected (no GPU needed)."""
import pytest


@pytest.fixture(scope="module")
def px():
    import paper_2602_10141_b300 as px
    return px


def test_corrupt_checkpoint_rejected(px, tmp_path):
    ck = tmp_path / "bad.ckpt"
    ck.write_text("permx-schur-ckpt 1\nn 19\nprimes 3 1 2 3\ndone 0\ncursor 0 0\nsum 0000000000000000\n")
    with pytest.raises(px.PermxError) as e:
        px.perm_schur_crt_ex(19, 0, str(ck))
    assert e.value.code == px.PERMX_EIO
    ck.write_text("garbage")
    with pytest.raises(px.PermxError) as e:
        px.perm_schur_crt_ex(19, 0, str(ck))
    assert e.value.code == px.PERMX_EIO


def test_checkpoint_from_other_run_rejected(px, tmp_path):
    # a well-formed file (valid FNV-1a checksum) written for n = 17 is refused for n = 19
    body = "permx-schur-ckpt 2\nn 17\nprimes 2 2147483647 2147483629\ndone 0\ncursor 0 0\n"
    h = 1469598103934665603
    for c in body.encode():
        h ^= c
        h = (h * 1099511628211) % (1 << 64)
    ck = tmp_path / "other.ckpt"
    ck.write_text(body + "sum %016x\n" % h)
    with pytest.raises(px.PermxError) as e:
        px.perm_schur_crt_ex(19, 0, str(ck))
    assert e.value.code == px.PERMX_EINVAL
    assert "different run" in px.last_error()


def test_unreadable_checkpoint_path_is_an_error(px, tmp_path):
    """A checkpoint path that cannot be opened for a reason other than 'no such
    file' (here a regular file used as a directory) is an I/O error, reported
    before any GPU work, not a fresh start."""
    f = tmp_path / "plain_file"
    f.write_text("x")
    with pytest.raises(px.PermxError) as e:
        px.perm_schur_crt_ex(19, 0, str(f / "run.ckpt"))
    assert e.value.code == px.PERMX_EIO
    assert "cannot read checkpoint" in px.last_error()


def _ckpt(body: str) -> str:
    h = 1469598103934665603
    for c in body.encode():
        h ^= c
        h = (h * 1099511628211) % (1 << 64)
    return body + "sum %016x\n" % h


def test_checkpoint_with_impossible_state_rejected(px, tmp_path):
    """A checkpoint with a valid checksum and matching run, but a cursor at or
    past the end of the walk (2^(n-1) Gray indices), a partial sum or a
    finished residue not below its prime, is an I/O error before any GPU work;
    such a cursor would otherwise never advance."""
    n = 19
    k = px.perm_schur_prime_count(n)
    primes = px.perm_primes_1_mod_n(n, k + 1)
    head = "permx-schur-ckpt 2\nn %d\nprimes %d %s\n" % (n, len(primes), " ".join(map(str, primes)))
    cases = {
        "cursor": head + "done 0\ncursor %d 0\n" % (1 << (n - 1)),
        "partial": head + "done 0\ncursor 4096 %d\n" % primes[0],
        "residue": head + "done 1 %d\ncursor 0 0\n" % primes[0],
    }
    for what, body in cases.items():
        ck = tmp_path / f"{what}.ckpt"
        ck.write_text(_ckpt(body))
        with pytest.raises(px.PermxError) as e:
            px.perm_schur_crt_ex(n, 0, str(ck))
        assert e.value.code == px.PERMX_EIO, what
