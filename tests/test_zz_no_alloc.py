"""perm_modp_noalloc, the entry point for callers that cannot allocate memory
during a call (another allocator owns the device budget, or the call sits on
a path that must not enter an allocator).  Called through the C-ABI and
checked bit-for-bit against perm_modp, the allocating batched entry point,
on two calls in a row that reuse the same fixed scratch array.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _batch(seed, sizes, primes):
    g = np.random.default_rng(seed)
    mats = [g.integers(0, p, (k, k), dtype=np.uint64).astype(np.uint32) for k, p in zip(sizes, primes)]
    n = np.array(sizes, np.int32)
    off = np.concatenate([[0], np.cumsum([k * k for k in sizes])[:-1]]).astype(np.int64)
    flat = np.concatenate([m.reshape(-1) for m in mats]).astype(np.uint32)
    return flat, n, off, np.array(primes, np.uint32)


def _call(lib_fn, dA, n, off, p, out, stream):
    P = ctypes.POINTER
    return lib_fn(ctypes.c_void_p(dA.data_ptr()), n.ctypes.data_as(P(ctypes.c_int32)),
                  off.ctypes.data_as(P(ctypes.c_int64)), p.ctypes.data_as(P(ctypes.c_uint32)),
                  ctypes.c_int64(len(n)), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_allocating_path_twice():
    import torch

    import paper_2602_10141_b300 as px
    lib = px._lib
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        # ragged sizes, several primes, n up to the F_p maximum of 48 (Gray walk truncated
        # only by n: n = 48 would take minutes, so the large end stays at 30)
        _batch(1, [5, 12, 30, 1, 17, 12, 24, 9], [2147483629, 2147483647, 1000003, 65537, 2147483629, 3, 97, 2147483647]),
        # a second, different batch: the fixed scratch must hold nothing of the first call
        _batch(2, [26, 3, 3, 20, 14] + [8] * 59, [2147483647] * 64),
    ]
    for flat, n, off, p in cases:
        dA = torch.from_numpy(flat.view(np.int32)).cuda()
        ref = torch.zeros(len(n), dtype=torch.int32, device="cuda")
        got = torch.full((len(n),), -1, dtype=torch.int32, device="cuda")
        assert _call(lib.perm_modp, dA, n, off, p, ref, stream) == 0, px.last_error()
        assert _call(lib.perm_modp_noalloc, dA, n, off, p, got, stream) == 0, px.last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_rejects_oversized_batch():
    import torch

    import paper_2602_10141_b300 as px
    flat, n, off, p = _batch(3, [4] * 65, [2147483629] * 65)
    dA = torch.from_numpy(flat.view(np.int32)).cuda()
    out = torch.zeros(65, dtype=torch.int32, device="cuda")
    rc = _call(px._lib.perm_modp_noalloc, dA, n, off, p, out, torch.cuda.current_stream().cuda_stream)
    assert rc == px.PERMX_EINVAL
    assert "PERMX_NOALLOC_MAX_BATCH" in px.last_error()


def test_noalloc_and_batched_take_entries_mod_p():
    """Residues at or above p are taken mod p while staging, on both entry
    points: the result is the oracle's permanent of A mod p."""
    import torch

    import oracle as O
    import paper_2602_10141_b300 as px
    lib = px._lib
    stream = torch.cuda.current_stream().cuda_stream
    g = np.random.default_rng(11)
    sizes, primes = [5, 12, 9], [2147483629, 65537, 13]
    raw = [g.integers(0, 1 << 32, (k, k), dtype=np.uint64).astype(np.uint32) for k in sizes]
    raw[0] = (raw[0].astype(np.uint64) % primes[0] + primes[0]).astype(np.uint32)   # every entry in [p, 2p)
    n = np.array(sizes, np.int32)
    off = np.concatenate([[0], np.cumsum([k * k for k in sizes])[:-1]]).astype(np.int64)
    flat = np.concatenate([m.reshape(-1) for m in raw]).astype(np.uint32)
    p = np.array(primes, np.uint32)
    want = [O.perm_modp_dp((m.astype(np.uint64) % q).astype(np.uint32), q) for m, q in zip(raw, primes)]
    dA = torch.from_numpy(flat.view(np.int32)).cuda()
    for fn in (lib.perm_modp, lib.perm_modp_noalloc):
        out = torch.full((3,), -1, dtype=torch.int32, device="cuda")
        assert _call(fn, dA, n, off, p, out, stream) == 0, px.last_error()
        torch.cuda.synchronize()
        assert [int(x) & 0xFFFFFFFF for x in out.cpu().numpy()] == want
