"""Continuous-batching server (serve_*): results equal the batched path bit for
bit whether a request runs alone or in a mix, requests admitted while others
run overlap with them, and admission limits behave."""
import time

import numpy as np
import pytest

import oracle as O
from workloads import ensemble, geodesic_cycle, random_residues, rng

pytestmark = pytest.mark.gpu


class Server:
    """Test adapter over the binding's Server: calls return the C-ABI codes
    instead of raising, so the tests can check error paths."""

    def __init__(self, px, **cfg):
        self.px = px
        self.S = px.Server(**cfg)
        self.lib, self.h = px._lib, self.S.h

    def submit(self, A, field, p=0):
        try:
            return 0, self.S.submit(A, field, p)
        except self.px.PermxError as e:
            return e.code, 0

    def poll(self, ticket, field):
        try:
            r = self.S.poll(ticket)
        except self.px.PermxError as e:
            return e.code, None, None
        if r is None:
            return 0, None, None
        return 0, r[0], r[1]

    def wait(self, tickets, timeout=120.0):
        out = {}
        t0 = time.time()
        while len(out) < len(tickets):
            for t, f in tickets:
                if t in out:
                    continue
                rc, v, lat = self.poll(t, f)
                assert rc == 0, self.px.last_error()
                if v is not None:
                    out[t] = (v, lat)
            assert time.time() - t0 < timeout
            time.sleep(0.0005)
        return out

    def stats(self):
        st = self.S.stats()
        return [st[k] for k in ("submitted", "completed", "resident", "steps", "launches")]

    def close(self):
        self.S.close()


def _batched(px, A, field, p=0):
    import torch
    if field == 2:
        o = torch.empty(1, dtype=torch.int32, device="cuda")
        px.perm_modp(torch.from_numpy(np.ascontiguousarray(A).view(np.int32).reshape(-1)).cuda(), [A.shape[0]], [0],
                     [p], o)
        torch.cuda.synchronize()
        return int(o.cpu().numpy()[0]) & 0xFFFFFFFF
    cplx = field == 0
    o = torch.empty(1, dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    (px.perm_c128 if cplx else px.perm_f64)(torch.from_numpy(A.reshape(-1)).cuda(), [A.shape[0]], [0], o)
    torch.cuda.synchronize()
    return complex(o.cpu().numpy()[0]) if cplx else float(o.cpu().numpy()[0])


@pytest.fixture(scope="module")
def px():
    import paper_2602_10141_b300 as px
    return px


def _mix(seed, count):
    g = rng(seed)
    reqs = []
    for i in range(count):
        kind = i % 4
        if kind == 0:
            n = int(g.integers(10, 17))
            reqs.append((ensemble("haar_u", n, 1, seed=seed * 1000 + i)[0], 0, 0))
        elif kind == 1:
            n = int(g.integers(10, 17))
            reqs.append((ensemble("goe", n, 1, seed=seed * 1000 + i)[0], 1, 0))
        elif kind == 2:
            n = int(g.choice([9, 11, 13, 15]))
            t = int(g.integers(0, 201)) / 200
            reqs.append((geodesic_cycle(n, t, "principal").astype(np.complex128), 0, 0))
        else:
            n = int(g.integers(16, 21))
            p = O.primes_1_mod_n(n, 1)[0]
            reqs.append((random_residues(n, p, g), 2, p))
    return reqs


@pytest.mark.parametrize("plain", [0, 1])
def test_mixed_requests_equal_batched_path(px, plain):
    S = Server(px, plain_fifo=plain)
    try:
        reqs = _mix(7, 40)
        tickets = []
        for A, f, p in reqs:
            rc, t = S.submit(A, f, p)
            assert rc == 0, px.last_error()
            tickets.append((t, f))
        res = S.wait(tickets)
        for (A, f, p), (t, _) in zip(reqs, tickets):
            v = res[t][0]
            assert v == _batched(px, A, f, p), (A.shape[0], f)
        # spot-check against the oracle
        A, f, p = reqs[3]
        assert res[tickets[3][0]][0] == O.perm_modp_dp(A, p)
        A, f, p = reqs[0]
        ref = O.perm_dp(A)
        assert abs(res[tickets[0][0]][0] - ref) <= 1e-9 * abs(ref)
    finally:
        S.close()


def test_fp64_mode_server_equals_batched_path(px):
    """A server created in FP64 mode keeps the double-double partial slots and
    finalisation; its results equal the FP64-mode batched path bit for bit and
    the oracle within the tolerance."""
    old = px.permx_set_fp_arith(px.FP_ARITH_FP64)
    S = None
    try:
        S = Server(px)
        reqs = [r for r in _mix(11, 24) if r[1] != 2]
        tickets = []
        for A, f, p in reqs:
            rc, t = S.submit(A, f, p)
            assert rc == 0, px.last_error()
            tickets.append((t, f))
        res = S.wait(tickets)
        for (A, f, p), (t, _) in zip(reqs, tickets):
            v = res[t][0]
            assert v == _batched(px, A, f, p), (A.shape[0], f)
        for (A, f, p), (t, _) in list(zip(reqs, tickets))[:4]:
            ref = O.perm_dp(A)
            assert abs(res[t][0] - ref) <= 1e-9 * max(abs(ref), 1e-12), (A.shape[0], f)
    finally:
        if S is not None:
            S.close()
        px.permx_set_fp_arith(old)


def test_arrivals_join_while_others_run(px):
    # a long request is admitted first; short ones submitted while it runs join at the
    # next step and finish before it (continuous batching, not a FIFO queue)
    S = Server(px)
    try:
        big = ensemble("haar_u", 29, 1, seed=9)[0]
        rc, tb = S.submit(big, 0)
        assert rc == 0
        time.sleep(0.005)
        small = [ensemble("haar_u", 12, 1, seed=100 + i)[0] for i in range(20)]
        ts = []
        for A in small:
            rc, t = S.submit(A, 0)
            assert rc == 0
            ts.append((t, 0))
        res = S.wait(ts + [(tb, 0)])
        lat_big = res[tb][1]
        assert max(res[t][1] for t, _ in ts) < lat_big - 0.005
        assert res[tb][0] == _batched(px, big, 0)
        for A, (t, _) in zip(small, ts):
            assert res[t][0] == _batched(px, A, 0)
        st = S.stats()
        assert st[0] == st[1] == 21 and st[3] >= 2
    finally:
        S.close()


def test_memory_bound_admission_and_limits(px):
    # a device budget that holds only a few requests at once still completes all of them
    S = Server(px, device_bytes=1 << 13, max_requests=8)
    try:
        reqs = [ensemble("ginibre_c", 14, 1, seed=200 + i)[0] for i in range(8)]
        ts = []
        for A in reqs:
            rc, t = S.submit(A, 0)
            assert rc == 0
            ts.append((t, 0))
        rc, _ = S.submit(reqs[0], 0)
        assert rc == px.PERMX_EBUSY
        res = S.wait(ts)
        for A, (t, _) in zip(reqs, ts):
            assert res[t][0] == _batched(px, A, 0)
        rc, _, _ = S.poll(123456789, 0)
        assert rc == px.PERMX_ENOTFOUND
        rc, _ = S.submit(np.zeros((3, 3), np.uint32) + 7, 2, 7)
        assert rc == px.PERMX_EINVAL   # entries must be below p
    finally:
        S.close()


def test_nonfinite_request_gives_nan_and_leaves_others(px):
    """A served matrix with a NaN or infinite entry yields NaN (integer mode),
    and the requests served beside it keep their batched-path bits."""
    old = px.permx_set_fp_arith(px.FP_ARITH_INT)
    S = Server(px)
    try:
        good = [(ensemble("haar_u", 12, 1, seed=900)[0], 0), (ensemble("goe", 14, 1, seed=901)[0], 1)]
        bad_c = ensemble("haar_u", 13, 1, seed=902)[0].copy()
        bad_c[2, 3] = complex(np.nan, 0.0)
        bad_r = ensemble("goe", 11, 1, seed=903)[0].copy()
        bad_r[0, 0] = np.inf
        reqs = [good[0], (bad_c, 0), good[1], (bad_r, 1)]
        tickets = []
        for A, f in reqs:
            rc, t = S.submit(A, f)
            assert rc == 0, px.last_error()
            tickets.append((t, f))
        res = S.wait(tickets)
        vals = [res[t][0] for t, _ in tickets]
        assert vals[0] == _batched(px, good[0][0], 0)
        assert vals[2] == _batched(px, good[1][0], 1)
        assert np.isnan(vals[1].real) and np.isnan(vals[1].imag)
        assert np.isnan(vals[3])
    finally:
        S.close()
        px.permx_set_fp_arith(old)


def test_drain_reports_timeout_then_completes(px):
    """serve_drain returns PERMX_ETIMEOUT while a long request is in flight and
    0 once everything has finished; the result is still the batched one."""
    S = Server(px)
    try:
        n = 29
        p = O.primes_1_mod_n(n, 1)[0]
        A = random_residues(n, p, rng(77))            # 2^28 Gray steps: milliseconds on the GPU
        rc, t = S.submit(A, 2, p)
        assert rc == 0, px.last_error()
        assert S.lib.serve_drain(S.h, 0) == px.PERMX_ETIMEOUT
        assert S.lib.serve_drain(S.h, 60_000) == 0, px.last_error()
        res = S.wait([(t, 2)])
        assert res[t][0] == _batched(px, A, 2, p)
    finally:
        S.close()


def _block_diag(blocks):
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n), dtype=blocks[0].dtype)
    o = 0
    for b in blocks:
        k = b.shape[0]
        M[o:o + k, o:o + k] = b
        o += k
    return M


def test_max_size_requests_served_with_small_ones(px):
    """The largest float (n = 32, complex) and a large F_p request (n = 40)
    served beside small requests: block-diagonal matrices with rows and
    columns shuffled, so the oracle's value is the product of the blocks'
    permanents; the served results also equal the batched path's."""
    g = rng(5000)
    S = Server(px)
    try:
        cb = [ensemble("haar_u", 8, 1, seed=5000 + k)[0] for k in range(4)]
        C = _block_diag(cb)
        P, Q = g.permutation(32), g.permutation(32)
        C = np.ascontiguousarray(C[P][:, Q])
        c_ref = np.prod([O.perm_dp(b) for b in cb])
        p = 2147483629
        mb = [random_residues(10, p, g) for _ in range(4)]
        M = _block_diag(mb).astype(np.uint32)
        P, Q = g.permutation(40), g.permutation(40)
        M = np.ascontiguousarray(M[P][:, Q])
        m_ref = 1
        for b in mb:
            m_ref = m_ref * O.perm_modp_dp(b, p) % p
        small = [ensemble("goe", 11, 1, seed=5100 + i)[0] for i in range(8)]
        rc, tc = S.submit(C, 0)
        assert rc == 0, px.last_error()
        rc, tm = S.submit(M, 2, p)
        assert rc == 0, px.last_error()
        ts = []
        for A in small:
            rc, t = S.submit(A, 1)
            assert rc == 0
            ts.append((t, 1))
        res = S.wait([(tc, 0), (tm, 2)] + ts, timeout=300.0)
        assert abs(res[tc][0] - c_ref) <= 1e-9 * abs(c_ref), (res[tc][0], c_ref)
        assert res[tc][0] == _batched(px, C, 0)
        assert res[tm][0] == m_ref
        for A, (t, _) in zip(small, ts):
            assert res[t][0] == _batched(px, A, 1)
    finally:
        S.close()


def test_work_budget_admission_lets_small_requests_pass(px):
    """Admission by outstanding work: with a budget that holds one large
    request, the second large one waits until the first one's steps have run,
    while small requests queued behind it are admitted and finish first;
    every result equals the batched path's."""
    big = [ensemble("haar_u", 26, 1, seed=600 + i)[0] for i in range(2)]
    cost_big = 26 * 2 ** 25                           # complex128-term equivalents of one n = 26 walk
    S = Server(px, work_budget=cost_big + cost_big // 2)
    try:
        tb = []
        for A in big:
            rc, t = S.submit(A, 0)
            assert rc == 0, px.last_error()
            tb.append((t, 0))
        small = [ensemble("goe", 12, 1, seed=700 + i)[0] for i in range(16)]
        ts = []
        for A in small:
            rc, t = S.submit(A, 1)
            assert rc == 0
            ts.append((t, 1))
        res = S.wait(tb + ts)
        # the second large request starts only after the first one's work has run
        assert res[tb[1][0]][1] > res[tb[0][0]][1]
        assert max(res[t][1] for t, _ in ts) < res[tb[1][0]][1]
        for A, (t, _) in zip(big, tb):
            assert res[t][0] == _batched(px, A, 0)
        for A, (t, _) in zip(small, ts):
            assert res[t][0] == _batched(px, A, 1)
        st = S.S.stats()
        assert st["completed"] == 18 and st["pending"] == 0 and st["resident"] == 0
        assert st["resident_work"] == 0
        assert 0.0 < st["gpu_busy_ms"] <= st["uptime_ms"]
    finally:
        S.close()


def test_unlimited_and_tiny_budgets_give_the_same_bits(px):
    """The work budget changes only when requests run, never their results:
    an unlimited budget and one smaller than any request (one request
    resident at a time) serve a mixed trace bit-identically."""
    reqs = _mix(11, 24)
    out = []
    for budget in (-1, 1):
        S = Server(px, work_budget=budget)
        try:
            tickets = []
            for A, f, p in reqs:
                rc, t = S.submit(A, f, p)
                assert rc == 0, px.last_error()
                tickets.append((t, f))
            res = S.wait(tickets)
            out.append([res[t][0] for t, _ in tickets])
        finally:
            S.close()
    assert out[0] == out[1]
