"""perm_sample_stats on the GPU: parity with the oracle's sample statistics on
seeded inputs (counts, minima and maxima exact, moments to rounding), the
argument checks, and end-to-end checks of batches of permanents (batched GPU
walk + GPU statistics) against what the mathematics and the paper fix:

* E|perm U|^2 = n! (n-1)! / (2n-1)! for Haar U(n) (Schur orthogonality on
  the symmetric power; the paper's n!/n^n is a different number), and the
  exponential law of |perm U|^2 (paper §3.2, eq. "exp"), which together give
  the paper's 18 % anti-concentration probability at n = 17 (§7);
* circularity E[perm(U)^2] ~ 0 (§3.2);
* Var and excess kurtosis of perm(O), Haar O(n) (§5.1, Table "orthogonal");
* perm(H) real for Hermitian H (§6.1, Proposition "herm-real");
* skewness and excess kurtosis of log|perm| (§7, Table "lognormal");
* Pr[|perm|^2 >= E/n^2], E = n! sigma^(2n), for the Gaussian ensembles (§7).

The statistical checks use 50,000 samples (the paper's sample size) from
fixed seeds; their tolerances are several standard errors of the difference
between two such estimates."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from workloads import rng
from workloads.device import batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def px():
    import paper_2602_10141_b300 as px
    return px


MOMENTS = ["mean_re", "mean_im", "var_re", "var_im", "cov_re_im", "skew_re", "exkurt_re", "mean_abs2",
           "mean_abs4", "mean_z2_re", "mean_z2_im", "log_mean", "log_var", "log_skew", "log_exkurt"]
EXACT = ["count", "count_nonzero", "count_above", "count_real", "min_abs2", "max_abs2"]


def _compare(got, ref, scale_re, scale_log):
    for k in EXACT:
        assert got[k] == ref[k], (k, got[k], ref[k])
    # each moment against its own natural scale (a mean near 0 is compared with the spread)
    scales = {"mean_re": scale_re, "mean_im": scale_re, "cov_re_im": ref["var_re"] + ref["var_im"],
              "mean_z2_re": ref["mean_abs2"], "mean_z2_im": ref["mean_abs2"], "log_mean": scale_log,
              "skew_re": 1.0, "log_skew": 1.0}
    for k in MOMENTS:
        r, g = ref[k], got[k]
        if math.isnan(r):
            assert math.isnan(g), k
            continue
        s = max(abs(r), scales.get(k, abs(r)), 1e-300)
        assert abs(g - r) <= 1e-11 * s, (k, g, r)


def _values(kind, count, g):
    if kind == "complex":
        v = g.normal(0.2, 1.0, count) + 1j * g.normal(-0.1, 0.7, count)
    elif kind == "real":
        v = g.standard_cauchy(count)          # heavy tails, like the Gaussian-ensemble permanents
    else:                                     # tiny Haar-like magnitudes with zeros and exact ties
        v = (g.normal(size=count) + 1j * g.normal(size=count)) * 1e-5
        v[::97] = 0.0
        v[1::89] = 0.5e-5 + 0j
    return v


@pytest.mark.parametrize("count", [1, 7, 2049, 100_003, 3_000_001])
@pytest.mark.parametrize("kind", ["complex", "real", "tiny"])
def test_parity_with_oracle(px, kind, count):
    import torch
    g = rng(1000 + count)
    v = _values(kind, count, g)
    thr = 0.25e-10 if kind == "tiny" else 0.9
    tol = 0.0 if kind == "tiny" else 0.3          # 0: the exactly-real test
    ref = O.sample_stats(v, threshold=thr, real_tol=tol)
    dt = torch.complex128 if np.iscomplexobj(v) else torch.float64
    got = px.perm_sample_stats(torch.from_numpy(v).to(dtype=dt).cuda(), threshold=thr, real_tol=tol)
    spread = math.sqrt(ref["var_re"] + ref["var_im"]) or 1.0
    _compare(got, ref, spread, math.sqrt(ref["log_var"]) if ref["log_var"] == ref["log_var"] else 1.0)


def test_deterministic_and_async(px):
    import torch
    v = torch.from_numpy(_values("complex", 123_457, rng(3))).cuda()
    a = px.perm_sample_stats(v, threshold=1.0)
    s = torch.cuda.Stream()
    out = torch.empty(256, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(s):
        px.perm_sample_stats_async(v, out, threshold=1.0, stream=s)
    s.synchronize()
    b = px.PermStats.from_buffer_copy(out[:168].cpu().numpy().tobytes()).as_dict()
    assert a == b or all((a[k] == b[k]) or (a[k] != a[k] and b[k] != b[k]) for k in a)


def test_argument_errors(px):
    import torch
    v = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(px.PermxError):
        px.perm_sample_stats_async(v[:0], out)
    with pytest.raises(px.PermxError):
        px.perm_sample_stats_async(v, out, real_tol=-1.0)
    # misaligned complex values (8-byte offset)
    raw = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(px.PermxError):
        px._check(px._lib.perm_sample_stats(px.FIELD_C128, raw.data_ptr() + 8, 4, 1.0, 0.0, out.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream))
    with pytest.raises(px.PermxError):
        px._check(px._lib.perm_sample_stats(px.FIELD_MODP, raw.data_ptr(), 4, 1.0, 0.0, out.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream))


# ---------------------------------------------------------------------------
# batches of permanents: GPU walk + GPU statistics
# ---------------------------------------------------------------------------

N_SAMPLES = 50_000


def _perms(px, name, n, count=N_SAMPLES, seed=0):
    import torch
    A = batch(name, n, count, seed)
    out = torch.empty(count, dtype=A.dtype, device="cuda")
    f = px.perm_c128 if A.dtype == torch.complex128 else px.perm_f64
    f(A.reshape(-1), np.full(count, n, np.int32), np.arange(count, dtype=np.int64) * n * n, out)
    return out


def _haar_m2(n):
    return math.factorial(n) * math.factorial(n - 1) / math.factorial(2 * n - 1)


@pytest.mark.parametrize("n", [7, 11, 17])
def test_haar_unitary_second_moment_and_circularity(px, n):
    v = _perms(px, "haar_u", n, seed=n)
    thr = math.factorial(n) / n ** n / n ** 2          # the paper's E/n^2 with E = n!/n^n
    s = px.perm_sample_stats(v, threshold=thr, real_tol=1e-6)
    mu = _haar_m2(n)
    se = math.sqrt(max(s["mean_abs4"] - s["mean_abs2"] ** 2, 0.0) / N_SAMPLES)
    assert abs(s["mean_abs2"] - mu) <= 4 * se, (s["mean_abs2"], mu, se)
    # exponential law: E|z|^4 = 2 (E|z|^2)^2
    assert abs(s["mean_abs4"] / s["mean_abs2"] ** 2 - 2.0) <= 0.15
    # circular: E z^2 ~ 0, Re and Im uncorrelated with equal variances
    assert math.hypot(s["mean_z2_re"], s["mean_z2_im"]) <= 0.03 * s["mean_abs2"]
    assert abs(s["var_re"] / s["var_im"] - 1) <= 0.04
    assert abs(s["cov_re_im"]) <= 0.03 * s["mean_abs2"]
    frac = s["count_above"] / N_SAMPLES
    pred = math.exp(-thr / mu)
    assert abs(frac - pred) <= 4 * math.sqrt(pred * (1 - pred) / N_SAMPLES) + 1e-3, (frac, pred)
    if n == 17:
        assert abs(frac - 0.18) <= 0.015                 # paper §7: 18 % at n = 17
    assert s["count_real"] <= 0.01 * N_SAMPLES          # a generic complex permanent is not real
    # the exponential law itself: empirical CDF of |perm U|^2 / mu (device histogram on
    # geometric edges) within a few 1/sqrt(N) of 1 - exp(-x)
    tq = np.geomspace(1e-3, 12.0, 64)
    h = px.perm_sample_histogram(v, tq * mu, px.HIST_ABS2)
    assert h.sum() == N_SAMPLES
    dev = np.max(np.abs(np.cumsum(h)[:-1] / N_SAMPLES - (1.0 - np.exp(-tq))))
    assert dev <= (0.03 if n == 7 else 0.015), dev


# paper §5.1, Table "orthogonal" (tests/golden/orthogonal_table.txt): n, Var[perm(O)], excess kurtosis;
# n = 17, 19 are reported by the bench, not tested (kurtosis differences of ~0.1 are within sampling)
ORTHOGONAL = [(int(r[0]), float(r[1]), float(r[2])) for r in read_golden("orthogonal_table.txt")][:3]


@pytest.mark.parametrize("n,var,kurt", ORTHOGONAL)
def test_haar_orthogonal_table(px, n, var, kurt):
    s = px.perm_sample_stats(_perms(px, "haar_o", n, seed=100 + n))
    assert abs(s["var_re"] / var - 1) <= 0.05, (s["var_re"], var)
    assert abs(s["exkurt_re"] - kurt) <= 0.15, (s["exkurt_re"], kurt)
    assert abs(s["mean_re"]) <= 4 * math.sqrt(s["var_re"] / N_SAMPLES)
    assert s["count_real"] == N_SAMPLES


@pytest.mark.parametrize("name", ["gue", "haar_u_control"])
def test_hermitian_permanents_are_real(px, name):
    n = 11
    v = _perms(px, "gue" if name == "gue" else "haar_u", n, count=20_000, seed=7)
    s = px.perm_sample_stats(v, real_tol=1e-9)
    if name == "gue":
        assert s["count_real"] == 20_000
    else:
        assert s["count_real"] == 0


# paper §7.2, Table "lognormal" (tests/golden/lognormal_table.txt): (ensemble, n) -> (skew, excess
# kurtosis) of log|perm|; the n = 7 rows of every ensemble and Ginibre-C at n = 13
LOGNORMAL = [(r[0], int(r[1]), float(r[2]), float(r[3])) for r in read_golden("lognormal_table.txt")
             if r[1] == "7" or (r[0] == "ginibre_c" and r[1] == "13")]


@pytest.mark.parametrize("name,n,skew,kurt", LOGNORMAL)
def test_log_moments_table(px, name, n, skew, kurt):
    s = px.perm_sample_stats(_perms(px, name, n, seed=200 + n))
    assert s["count_nonzero"] == N_SAMPLES
    assert abs(s["log_skew"] - skew) <= 0.1, (s["log_skew"], skew)
    assert abs(s["log_exkurt"] - kurt) <= 0.3, (s["log_exkurt"], kurt)


def _entry_m2(name, n):
    """Mean E|h_ij|^2 over the entries: Ginibre 1; GUE 1/2 (diagonal N(0,1/2),
    off-diagonal CN(0,1/2)); GOE (n+1)/(2n) (diagonal N(0,1), off-diagonal N(0,1/2))."""
    return {"ginibre_c": 1.0, "ginibre_r": 1.0, "gue": 0.5, "goe": (n + 1) / (2 * n)}[name]


@pytest.mark.parametrize("name", ["gue", "goe", "ginibre_c", "ginibre_r"])
def test_gaussian_anticoncentration(px, name):
    """Paper §7: Pr[|perm|^2 >= E/n^2] is 67 %-98 % at n = 17 for the four
    Gaussian ensembles and increases with n.  E = n! sigma^(2n), the second
    moment for independent entries of variance sigma^2 (n! for Ginibre, and
    n!/n^n for Haar unitaries, where it gives the paper's 18 %)."""
    count = 20_000
    fracs = []
    for n in (7, 11, 13, 17):
        E = math.factorial(n) * _entry_m2(name, n) ** n
        s = px.perm_sample_stats(_perms(px, name, n, count=count, seed=300 + n), threshold=E / n ** 2)
        fracs.append(s["count_above"] / count)
    assert 0.65 <= fracs[-1] <= 0.99, fracs
    assert all(b > a for a, b in zip(fracs, fracs[1:])), fracs


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_histogram_parity_with_oracle(px, kind):
    """perm_sample_histogram equals the oracle's counts exactly: linear and
    geometric edges, values placed exactly on edges, NaN entries, a ragged count."""
    import torch
    g = rng(600 + kind)
    count = 200_003
    v = g.normal(0.0, 1.0, count) + 1j * g.normal(0.0, 1.0, count)
    edges_lin = np.linspace(-3.0, 3.0, 61)
    edges_geo = np.geomspace(1e-4, 30.0, 129)          # |z|^2 on a log scale
    edges = edges_geo if kind == 0 else edges_lin
    v[:50] = edges[10:60] if kind != 2 else 1j * edges[10:60]   # exactly on edges (|z|^2 for kind 0 below)
    if kind == 0:
        v[:50] = np.sqrt(edges[10:60])                 # |z|^2 = rn(x*x) may differ from the edge by an ulp
    v[50:53] = complex(np.nan, np.nan)
    v[53] = complex(np.nan, 0.5)                       # NaN only in Re: still counted for Im
    ref = O.sample_histogram(v, edges, kind)
    got = px.perm_sample_histogram(torch.from_numpy(v).cuda(), edges, kind)
    assert list(got) == list(ref)
    assert got.sum() == count - (3 if kind == 2 else 4)
    # float64 values: Im = 0
    r = v.real.copy()
    got_r = px.perm_sample_histogram(torch.from_numpy(r).cuda(), edges_lin, 1)
    assert list(got_r) == list(O.sample_histogram(r, edges_lin, 1))


def test_histogram_argument_errors(px):
    import torch
    v = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(px.PermxError):
        px.perm_sample_histogram(v, [1.0, 1.0])            # not strictly increasing
    with pytest.raises(px.PermxError):
        px.perm_sample_histogram(v, [0.0, np.nan])
    with pytest.raises(px.PermxError):
        px.perm_sample_histogram(v, [0.0, 1.0], kind=3)
    got = px.perm_sample_histogram(v[:0], [0.0, 1.0])       # empty input: all zero
    assert list(got) == [0, 0, 0]
