"""The batched path's chunk plan (paper §2.2 Gray-code blocks), checked on the
host against the rules the kernels rely on: every matrix planned once, Gray
ranges split into 2^log2_chunks chunks of 2^ell steps covering the
Nijenhuis-Wilf walk, staged blocks and partial slots contiguous and disjoint,
column blocks aligned for the kernels' 16-byte loads, slot counts equal to
the kernels' lane-group rule, float chunk lengths independent of the batch,
and small F_p batches shortened only as far as the rule allows."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def px():
    import paper_2602_10141_b300 as px
    f = px._lib.permx_plan_describe
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_int, P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_int64), ctypes.c_int32,
                  P(ctypes.c_int64), P(ctypes.c_int64)]
    f.restype = ctypes.c_int
    return px


COLS = ("n", "ell", "log2_chunks", "ld", "mat_stride", "col_off", "items", "partials_per_mat", "part_off", "x64",
        "nmats")


def describe(px, field, sizes):
    n = np.ascontiguousarray(np.asarray(sizes, np.int32))
    g = np.zeros((64, len(COLS)), np.int64)
    order = np.zeros(len(n), np.int64)
    tot = np.zeros(2, np.int64)
    P = ctypes.POINTER
    k = px._lib.permx_plan_describe(field, n.ctypes.data_as(P(ctypes.c_int32)), len(n),
                                    g.ctypes.data_as(P(ctypes.c_int64)), 64, order.ctypes.data_as(P(ctypes.c_int64)),
                                    tot.ctypes.data_as(P(ctypes.c_int64)))
    assert k > 0, px.last_error()
    return [dict(zip(COLS, map(int, row))) for row in g[:k]], order, tot


def pad(n, q):
    return (n + q - 1) // q * q


def check_plan(px, field, sizes, pinned=()):
    groups, order, tot = describe(px, field, sizes)
    sizes = np.asarray(sizes)
    cplx, modp = field == px.FIELD_C128, field == px.FIELD_MODP
    # every matrix once, grouped by n in increasing order, batch order kept within a group
    assert sorted(order.tolist()) == list(range(len(sizes)))
    assert [g["n"] for g in groups] == sorted(set(sizes.tolist()))
    k = 0
    for g in groups:
        idx = order[k:k + g["nmats"]]
        assert (sizes[idx] == g["n"]).all() and (np.diff(idx) > 0).all()
        k += g["nmats"]
    col, part = 0, 0
    x64 = (not modp) and px.permx_get_fp_arith() == 1
    for g in groups:
        n = g["n"]
        # the Nijenhuis-Wilf walk: 2^(n-1) Gray steps per matrix, split into chunks
        assert g["ell"] >= 0 and g["log2_chunks"] >= 0 and g["ell"] + g["log2_chunks"] == n - 1
        # the walks count a chunk's steps modulo 2^(ell+1) in 32 bits
        assert g["ell"] <= 30
        assert g["items"] == g["nmats"] << g["log2_chunks"]
        # staged layout: n + 1 columns (the x column last) of ld entries
        ld = pad(n, 4) if modp else (pad(n, 2) if field == px.FIELD_F64 else n)
        assert g["ld"] == ld and g["x64"] == int(x64)
        words = 2 if cplx else 1
        assert g["mat_stride"] == (n + 1) * ld * words + (2 if g["x64"] else 0)
        assert g["col_off"] == col
        col += g["mat_stride"] * g["nmats"]
        # 16-byte loads: uint4 of residues, (long)long2 / double2 of float words
        q = 4 if modp else 2
        assert g["col_off"] % q == 0 and g["mat_stride"] % q == 0
        # partial slots: one per lane group of chunks, as the kernels number them
        lg = min(g["log2_chunks"], 4 if (g["x64"] and cplx and n >= 17) else 5)
        assert g["partials_per_mat"] == 1 << (g["log2_chunks"] - lg)
        assert g["part_off"] == part
        part += g["partials_per_mat"] * g["nmats"]
        if not modp:
            # float chunk lengths depend on (field, n) only, never on the batch
            assert g["ell"] == px.perm_tune_get(field, n)
        else:
            rule = px.perm_tune_get(field, n)
            assert min(n - 1, 5) <= g["ell"] <= rule or g["ell"] == rule
    assert tot[0] == col and tot[1] == part
    if modp:
        items = sum(g["items"] for g in groups)
        at_floor = all(g["ell"] <= min(g["n"] - 1, 5) or g["n"] in pinned for g in groups)
        assert items >= 1 << 18 or at_floor
    return groups


@pytest.mark.parametrize("field", [0, 1, 2])
def test_plans_of_random_ragged_batches(px, field):
    g = np.random.default_rng(40 + field)
    max_n = 48 if field == px.FIELD_MODP else 32
    for batch in (1, 2, 7, 100, 3000):
        for _ in range(4):
            lo = int(g.integers(1, max_n + 1))
            sizes = g.integers(lo, min(max_n, lo + int(g.integers(0, 12))) + 1, batch)
            check_plan(px, field, sizes)


def test_float_chunking_is_batch_independent(px):
    """The same n gets the same chunks alone and in any mix (float results do
    not depend on batch composition)."""
    for field in (px.FIELD_C128, px.FIELD_F64):
        for n in (3, 8, 14, 17, 20, 23, 32):
            alone = check_plan(px, field, [n])[0]
            mixed = [g for g in check_plan(px, field, [8, n, 23] * 50 + [12]) if g["n"] == n][0]
            assert (alone["ell"], alone["log2_chunks"]) == (mixed["ell"], mixed["log2_chunks"])


def test_small_modp_batches_get_shorter_chunks(px):
    """A lone n = 20 matrix (2^19 Gray steps) is cut down to the 2^5-step floor;
    4096 of them already fill the GPU at the rule's length; a lone S_33-size
    matrix has 2^22 chunks at the rule's length and is left alone."""
    rule = px.perm_tune_get(px.FIELD_MODP, 20)
    one = check_plan(px, px.FIELD_MODP, [20])[0]
    many = check_plan(px, px.FIELD_MODP, [20] * 4096)[0]
    assert one["ell"] == 5 < many["ell"] == rule
    big = check_plan(px, px.FIELD_MODP, [33])[0]
    assert big["ell"] == px.perm_tune_get(px.FIELD_MODP, 33) and big["items"] >= 1 << 18


def test_pinned_chunk_length_is_kept(px):
    try:
        px.perm_tune_set(px.FIELD_MODP, 20, 12)
        g = check_plan(px, px.FIELD_MODP, [20], pinned={20})[0]
        assert g["ell"] == 12 and g["log2_chunks"] == 7
        px.perm_tune_set(px.FIELD_C128, 20, 6)
        g = check_plan(px, px.FIELD_C128, [20, 20])[0]
        assert g["ell"] == 6
    finally:
        px.perm_tune_set(px.FIELD_MODP, 20, 0)
        px.perm_tune_set(px.FIELD_C128, 20, 0)


def test_describe_rejects_bad_arguments(px):
    P = ctypes.POINTER
    n = np.array([5, 0], np.int32)
    g = np.zeros((4, len(COLS)), np.int64)
    o = np.zeros(2, np.int64)
    t = np.zeros(2, np.int64)
    args = (n.ctypes.data_as(P(ctypes.c_int32)), 2, g.ctypes.data_as(P(ctypes.c_int64)), 4,
            o.ctypes.data_as(P(ctypes.c_int64)), t.ctypes.data_as(P(ctypes.c_int64)))
    assert px._lib.permx_plan_describe(px.FIELD_MODP, *args) == px.PERMX_EINVAL
    n[1] = 49
    assert px._lib.permx_plan_describe(px.FIELD_MODP, *args) == px.PERMX_EINVAL
    n[1] = 33
    assert px._lib.permx_plan_describe(px.FIELD_F64, *args) == px.PERMX_EINVAL
    assert px._lib.permx_plan_describe(7, *args) == px.PERMX_EINVAL


def test_longest_chunks_fit_the_step_counter(px):
    """The longest chunk any plan may hold is 2^30 steps (the walks keep the Gray
    index modulo 2^(ell+1) in 32 bits): a pinned F_p length of 30 is kept, and
    the tuning table refuses anything longer."""
    try:
        px.perm_tune_set(px.FIELD_MODP, 48, 30)
        g = check_plan(px, px.FIELD_MODP, [48], pinned={48})[0]
        assert g["ell"] == 30 and g["log2_chunks"] == 17
        with pytest.raises(px.PermxError):
            px.perm_tune_set(px.FIELD_MODP, 48, 31)
    finally:
        px.perm_tune_set(px.FIELD_MODP, 48, 0)
    for n in range(1, 49):
        assert check_plan(px, px.FIELD_MODP, [n])[0]["ell"] <= 30
