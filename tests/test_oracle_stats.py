"""Pins of the oracle's sample statistics (oracle.sample_stats): the
definitions of sample mean, variance, skewness and excess kurtosis against
library routines (numpy / scipy.stats with bias=True) and closed forms
(two-point and equally spaced unit-circle samples), the counts on exact
boundaries, and planted mistakes that the pins must catch."""
import inspect
import math

import numpy as np
import pytest
import scipy.stats as st

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _pins(f):
    """Yield (name, ok) for the pin battery on the statistics function f."""
    g = np.random.default_rng(5)
    # two-point +-a about a shifted mean: var a^2, skew 0, excess kurtosis -2
    a, mu = 0.75, 3.0
    x = np.array([mu + a, mu - a] * 8)
    s = f(x)
    yield "two_point_mean", abs(s["mean_re"] - mu) <= 1e-15
    yield "two_point_var", abs(s["var_re"] - a * a) <= 1e-15
    yield "two_point_kurt", abs(s["exkurt_re"] + 2.0) <= 1e-13
    yield "two_point_skew", abs(s["skew_re"]) <= 1e-13
    # library routines on skewed data with a nonzero mean
    x = g.gamma(2.0, 1.5, 5000) + 0.3
    s = f(x)
    yield "var", abs(s["var_re"] / np.var(x) - 1) <= 1e-12
    yield "skew", abs(s["skew_re"] / st.skew(x, bias=True) - 1) <= 1e-11
    yield "kurt", abs(s["exkurt_re"] / st.kurtosis(x, fisher=True, bias=True) - 1) <= 1e-11
    yield "abs4", abs(s["mean_abs4"] / np.mean(x ** 4) - 1) <= 1e-12
    lx = np.log(np.abs(x))
    yield "log_mean", abs(s["log_mean"] - np.mean(lx)) <= 1e-13
    yield "log_var", abs(s["log_var"] / np.var(lx) - 1) <= 1e-12
    yield "log_skew", abs(s["log_skew"] / st.skew(lx, bias=True) - 1) <= 1e-10
    yield "log_kurt", abs(s["log_exkurt"] / st.kurtosis(lx, fisher=True, bias=True) - 1) <= 1e-10
    # complex: covariance of Re, Im and the pseudo-covariance E[z^2]
    z = g.normal(1.0, 2.0, 4000) + 1j * (0.5 * g.normal(size=4000))
    z = z + 0.3 * z.real * 1j
    s = f(z)
    c = np.cov(z.real, z.imag, bias=True)
    yield "var_im", abs(s["var_im"] / c[1, 1] - 1) <= 1e-12
    yield "cov", abs(s["cov_re_im"] / c[0, 1] - 1) <= 1e-12
    yield "z2", abs(complex(s["mean_z2_re"], s["mean_z2_im"]) - np.mean(z * z)) <= 1e-12 * np.mean(np.abs(z) ** 2)
    yield "abs2", abs(s["mean_abs2"] / np.mean(np.abs(z) ** 2) - 1) <= 1e-12
    # N equally spaced points on the unit circle: E z = E z^2 = 0, var Re = var Im = 1/2
    N = 1000
    u = np.exp(2j * np.pi * np.arange(N) / N)
    s = f(u)
    yield "circle_mean", abs(s["mean_re"]) <= 1e-15 and abs(s["mean_im"]) <= 1e-15
    yield "circle_z2", abs(s["mean_z2_re"]) <= 1e-15 and abs(s["mean_z2_im"]) <= 1e-15
    yield "circle_var", abs(s["var_re"] - 0.5) <= 1e-15 and abs(s["var_im"] - 0.5) <= 1e-15
    # counts on exact boundaries: |z|^2 = 0.25 is counted at threshold 0.25;
    # z = 3 + 4i has |Im z| = 0.8 |z| exactly
    w = np.array([0.5, -0.5, 0.25, 0.0, 3 + 4j, 0.5j])
    s = f(w, threshold=0.25, real_tol=0.8)
    yield "above", s["count_above"] == 4
    yield "real", s["count_real"] == 5
    yield "nonzero", s["count_nonzero"] == 5
    yield "minmax", s["min_abs2"] == 0.0 and s["max_abs2"] == 25.0
    s = f(w, threshold=0.2500000000000001, real_tol=0.7999999999999999)
    yield "above_strict", s["count_above"] == 1
    yield "real_strict", s["count_real"] == 4


def test_sample_stats_pins():
    bad = [name for name, ok in _pins(O.sample_stats) if not ok]
    assert not bad, bad


def test_single_sample_and_all_zero():
    s = O.sample_stats(np.array([2.0]))
    assert s["var_re"] == 0.0 and math.isnan(s["exkurt_re"]) and s["log_mean"] == math.log(2.0)
    s = O.sample_stats(np.zeros(3, complex))
    assert s["count_nonzero"] == 0 and math.isnan(s["log_mean"])
    with pytest.raises(ValueError):
        O.sample_stats(np.array([]))


PLANTS = [
    ("central moments about 0 instead of the mean", "dr, di = re - mean_re, im - mean_im", "dr, di = re, im"),
    ("kurtosis not made excess", "/ np.float64(m2r) ** 2 - 3.0)", "/ np.float64(m2r) ** 2)"),
    ("skewness normalised by m2 instead of m2^1.5", "/ np.float64(m2r) ** 1.5)", "/ np.float64(m2r))"),
    ("variance divided by N - 1", "m2r = fs(dr * dr) / N", "m2r = fs(dr * dr) / (N - 1)"),
    ("pseudo-covariance sign", "fs(re * re - im * im)", "fs(re * re + im * im)"),
    ("threshold strict", "(a2 >= threshold)", "(a2 > threshold)"),
    ("real test against |z|^2", "real_tol * np.sqrt(a2)", "real_tol * a2"),
    ("log|z| without the 1/2", "logs = 0.5 * np.log(a2[nz])", "logs = np.log(a2[nz])"),
    ("log variance about 0", "dl = logs - lm", "dl = logs"),
]


@pytest.mark.parametrize("name,old,new", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_stats_mistake_is_caught(name, old, new):
    src = inspect.getsource(O.sample_stats)
    assert src.count(old) == 1, name
    ns = {"np": np, "math": math}
    exec(src.replace(old, new), ns)
    failed = [n for n, ok in _pins(ns["sample_stats"]) if not ok]
    assert failed, f"planted mistake '{name}' passed every pin"


def test_sample_histogram_pins():
    """Counts on exact edges, below and above, NaN skipped, |z|^2 and Re / Im
    selected; the total equals the non-NaN count; numpy's histogram on the
    interior bins agrees."""
    edges = [0.0, 0.25, 1.0, 4.0]
    z = np.array([0.5, -0.5, 0.25, 0.0, 3 + 4j, 0.5j, -2.0, 1.0, np.nan, 2j])
    # |z|^2: 0.25, 0.25, 0.0625, 0, 25, 0.25, 4, 1, nan, 4
    assert list(O.sample_histogram(z, edges, 0)) == [0, 2, 3, 1, 3]
    # Re z: 0.5, -0.5, 0.25, 0, 3, 0, -2, 1, (nan: skipped), 0
    assert list(O.sample_histogram(z, edges, 1)) == [2, 3, 2, 2, 0]
    # Im z: 0, 0, 0, 0, 4, 0.5, 0, 0, 0 (the NaN entry has imaginary part 0), 2
    assert list(O.sample_histogram(z, edges, 2)) == [0, 7, 1, 1, 1]
    g = np.random.default_rng(3)
    v = g.normal(size=5000) + 1j * g.normal(size=5000)
    e = np.linspace(-2.5, 2.5, 11)
    h = O.sample_histogram(v, e, 1)
    assert h.sum() == 5000
    ref, _ = np.histogram(v.real, bins=e)
    # numpy's bins are half-open except the last one, which is closed
    assert list(h[1:-2]) == list(ref[:-1]) and h[-2] <= ref[-1]


@pytest.mark.parametrize("name,old,new", [("edge goes to the lower bin", "e <= v", "e < v"),
                                          ("|z|^2 without Im", "re * re + im * im if kind == 0", "re * re if kind == 0")])
def test_planted_histogram_mistake_is_caught(name, old, new):
    src = inspect.getsource(O.sample_histogram)
    assert src.count(old) == 1, name
    ns = {"np": np}
    exec(src.replace(old, new), ns)
    f = ns["sample_histogram"]
    edges = [0.0, 0.25, 1.0, 4.0]
    z = np.array([0.5, -0.5, 0.25, 0.0, 3 + 4j, 0.5j, -2.0, 1.0, np.nan, 2j])
    ok = (list(f(z, edges, 0)) == [0, 2, 3, 1, 3] and list(f(z, edges, 1)) == [2, 3, 2, 2, 0])
    assert not ok, f"planted mistake '{name}' passed the pins"
