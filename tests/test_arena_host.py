"""The serving arena (admission by device memory) on the host, against an
independent model: blocks are 256-byte aligned and disjoint, allocation is
first-fit over the free gaps, the bytes in use and the largest free gap match
the model after every operation, freed neighbours merge (after releasing
everything one block spans the arena), and a request that no gap can hold is
refused."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def run():
    import paper_2602_10141_b300 as px
    f = px._lib.permx_arena_run
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_int64, P(ctypes.c_int64), ctypes.c_int32, P(ctypes.c_int64)]
    f.restype = ctypes.c_int

    def go(capacity, ops):
        o = np.ascontiguousarray(np.asarray(ops, np.int64).reshape(-1))
        res = np.zeros(3 * max(len(ops), 1), np.int64)
        k = f(capacity, o.ctypes.data_as(P(ctypes.c_int64)), len(ops), res.ctypes.data_as(P(ctypes.c_int64)))
        return k, res[:3 * len(ops)].reshape(-1, 3)
    return go


def rnd(x):
    return max(256, (x + 255) // 256 * 256)     # a zero-byte request still takes one 256-byte block


def gaps(live, capacity):
    """Free gaps [start, end) of [0, capacity) around the live blocks."""
    out, pos = [], 0
    for off, size in sorted(live.values()):
        if off > pos:
            out.append((pos, off))
        pos = max(pos, off + size)
    if capacity > pos:
        out.append((pos, capacity))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_arena_matches_first_fit_model(run, seed):
    g = np.random.default_rng(seed)
    capacity = int(g.choice([1 << 16, (1 << 20) + 100, 5000]))
    ops, live_ids = [], []
    for k in range(400):
        if live_ids and g.random() < 0.45:
            j = live_ids.pop(int(g.integers(0, len(live_ids))))
            ops.append((1, j))
        else:
            ops.append((0, int(g.integers(0, capacity // 6 + 2))))
            live_ids.append(k)
    # live_ids tracks requests, some of which the arena will refuse: a first
    # pass of the model finds those and turns their releases into requests
    model_ops, refused = [], set()
    live = {}
    for k, (kind, v) in enumerate(ops):
        if kind == 1 and v in refused:
            kind, v = 0, 0                    # replace by a small request (never released)
        model_ops.append((kind, v))
        if kind == 0:
            size = rnd(v)
            fit = [a for a, b in gaps(live, capacity) if b - a >= size]
            if fit:
                live[k] = (fit[0], size)
            else:
                refused.add(k)
        else:
            del live[v]
    # replay the cleaned sequence with the model checked after every operation
    nfree, res = run(capacity, model_ops)
    assert nfree >= 0
    live = {}
    for k, (kind, v) in enumerate(model_ops):
        if kind == 0:
            size = rnd(v)
            fit = [a for a, b in gaps(live, capacity) if b - a >= size]
            if fit:
                assert res[k, 0] == fit[0], (k, res[k, 0], fit[0])    # first fit
                assert res[k, 0] % 256 == 0 and res[k, 0] + size <= max(capacity, res[k, 0] + size)
                live[k] = (int(res[k, 0]), size)
            else:
                assert res[k, 0] == -1
        else:
            del live[v]
        spans = sorted(live.values())
        assert all(a + s <= b for (a, s), (b, _) in zip(spans, spans[1:]))      # disjoint
        assert res[k, 1] == sum(s for _, s in live.values())
        gl = [b - a for a, b in gaps(live, capacity)]
        assert res[k, 2] == (max(gl) if gl else 0)
    assert nfree == len(gaps(live, capacity))


def test_release_everything_merges_back(run):
    capacity = 1 << 20
    ops = [(0, 1000 * (k + 1)) for k in range(20)]
    order = np.random.default_rng(3).permutation(20)
    ops += [(1, int(j)) for j in order]
    nfree, res = run(capacity, ops)
    assert nfree == 1 and res[-1, 1] == 0 and res[-1, 2] == capacity


def test_oversized_request_refused(run):
    nfree, res = run(4096, [(0, 4097), (0, 4096), (0, 1)])
    assert res[0, 0] == -1 and res[1, 0] == 0 and res[2, 0] == -1 and nfree == 0


def test_bad_operations_rejected(run):
    import paper_2602_10141_b300 as px
    assert run(4096, [(1, 0)])[0] == px.PERMX_EINVAL            # release before any alloc
    assert run(4096, [(0, 10), (1, 0), (1, 0)])[0] == px.PERMX_EINVAL   # double release
    assert run(4096, [(0, 5000), (1, 0)])[0] == px.PERMX_EINVAL    # release of a refused block
    assert run(4096, [(2, 0)])[0] == px.PERMX_EINVAL
