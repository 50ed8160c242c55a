"""Planned batches and CUDA-graph replay (perm_plan_*) and the chunk-length
autotuner (perm_autotune / perm_tune_*): planned and replayed passes give
exactly the results of the one-shot batched calls."""
import numpy as np
import pytest

import oracle as O
from workloads import ensemble, random_residues, rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def px():
    import paper_2602_10141_b300 as px
    return px


def _pack(mats):
    n = [m.shape[0] for m in mats]
    off = np.concatenate([[0], np.cumsum([k * k for k in n])[:-1]]).astype(np.int64)
    return np.concatenate([m.reshape(-1) for m in mats]), n, off


def test_modp_plan_execute_and_graph(px):
    import torch
    g = rng(31)
    ps = [2147483629, 2147483647, 1000003]
    sizes = [5, 9, 17, 17, 22, 3, 12]
    mats = [random_residues(k, ps[i % 3], g) for i, k in enumerate(sizes)]
    primes = [ps[i % 3] for i in range(len(sizes))]
    flat, n, off = _pack(mats)
    A = torch.from_numpy(flat.astype(np.int32)).cuda()
    ref = torch.zeros(len(n), dtype=torch.int32, device="cuda")
    px.perm_modp(A, n, off, primes, ref)
    plan = px.Plan(px.FIELD_MODP, n, off, primes)
    try:
        out = torch.full((len(n),), -1, dtype=torch.int32, device="cuda")
        plan.execute(A, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        for _ in range(2):
            out.fill_(-1)
            plan.graph_launch(A, out)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        # new values in the same buffer: the replayed graph reads them
        mats2 = [random_residues(k, primes[i], g) for i, k in enumerate(sizes)]
        flat2, _, _ = _pack(mats2)
        A.copy_(torch.from_numpy(flat2.astype(np.int32)))
        plan.graph_launch(A, out)
        torch.cuda.synchronize()
        got = [int(x) & 0xFFFFFFFF for x in out.cpu().numpy()]
        assert got == [O.perm_modp_dp(m, p) for m, p in zip(mats2, primes)]
        # other buffers: the plan recaptures
        B = A.clone()
        out2 = torch.zeros_like(out)
        plan.graph_launch(B, out2)
        torch.cuda.synchronize()
        assert torch.equal(out2, out)
    finally:
        plan.close()


@pytest.mark.parametrize("cplx", [True, False])
def test_fp_plan_matches_one_shot(px, cplx):
    import torch
    name = "haar_u" if cplx else "goe"
    mats = [ensemble(name, k, 1, seed=40 + k)[0] for k in (6, 11, 16, 16, 19)]
    flat, n, off = _pack(mats)
    A = torch.from_numpy(flat).cuda()
    dt = torch.complex128 if cplx else torch.float64
    ref = torch.zeros(len(n), dtype=dt, device="cuda")
    (px.perm_c128 if cplx else px.perm_f64)(A, n, off, ref)
    plan = px.Plan(px.FIELD_C128 if cplx else px.FIELD_F64, n, off)
    try:
        out = torch.zeros_like(ref)
        plan.graph_launch(A, out)
        plan.graph_launch(A, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    finally:
        plan.close()


def test_autotune_keeps_results(px):
    import torch
    try:
        default = px.perm_tune_get(px.FIELD_MODP, 24)
        best = px.perm_autotune(px.FIELD_MODP, 24, 64, 2)
        assert 1 <= best <= 23 and abs(best - default) <= 3
        assert px.perm_tune_get(px.FIELD_MODP, 24) == best
        g = rng(5)
        p = 2147483629
        A = random_residues(24, p, g)
        out = torch.zeros(1, dtype=torch.int32, device="cuda")
        px.perm_modp(torch.from_numpy(A.astype(np.int32).reshape(-1)).cuda(), [24], [0], [p], out)
        assert int(out.item()) & 0xFFFFFFFF == O.perm_modp_dp(A, p)
        best_c = px.perm_autotune(px.FIELD_C128, 18, 32, 2)
        assert px.perm_tune_get(px.FIELD_C128, 18) == best_c
        U = ensemble("haar_u", 18, 1, seed=8)[0]
        o = torch.zeros(1, dtype=torch.complex128, device="cuda")
        px.perm_c128(torch.from_numpy(U.reshape(-1)).cuda(), [18], [0], o)
        ref = O.perm_dp(U)
        assert abs(complex(o.item()) - ref) <= 1e-9 * abs(ref)
    finally:
        px.perm_tune_set(px.FIELD_MODP, 24, 0)
        px.perm_tune_set(px.FIELD_C128, 18, 0)
    with pytest.raises(px.PermxError):
        px.perm_tune_set(7, 10, 3)
