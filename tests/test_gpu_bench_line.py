"""bench.py's default line on the GPU, at a small scale: one JSON line with
the headline keys of the bench contract, the roofline measured in the same
process, and the plain / batched / served objects each with its own clock
record and its comparison against one call per matrix or request."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_line_at_small_scale():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
                        "--no-cpu-baseline", "--extras-scale", "0.004"], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == "ryser_terms_per_s" and d["unit"] == "terms/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "schur_n33_fp_5primes" and d["config"]["perm_S33"] == "868088125376401545"
    ro = d["roofline"]
    assert ro["bound"] == "alu" and 0 < ro["frac"] < 1.2 and ro["peak"] > ro["achieved"] * 0.8
    assert set(ro["probe_rates_ops_per_s"]) == {"mul_wide_u32", "mad_lo_u32", "mul_hi_u32"}
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0 and d["gpu_launches"] > 0
    assert d["clocks"]["samples"] > 0
    p = d["plain"]
    assert p["value"] > 0 and p["batched_perms_per_s"] > p["value"] and p["max_rel_err_vs_oracle_sample"] < 1e-9
    assert p["clocks"]["sm_mhz"] is not None
    b = d["batched"]
    assert b["value"] > 0 and b["perms_per_step"] == 6 * 5 * 200 and b["max_rel_err_vs_oracle"] < 1e-9
    assert len(b["per_size"]) == 5 and all(r_["batched_perms_per_s"] > 0 for r_ in b["per_size"])
    assert len(b["tuned_chunk_log2"]) == 10 and b["clocks"]["sm_mhz"] is not None
    assert b["roofline"]["bound"] == "alu" and 0 < b["roofline"]["frac"] < 1.2
    assert b["fp64_roofline"]["frac"] > b["roofline"]["frac"]   # the integer walk outruns FP64
    s = d["served"]
    assert s["requests"] == 200 and s["continuous"]["p99_ms"] > 0 and s["plain_fifo"]["p99_ms"] > 0
    assert s["results_bit_identical_continuous_vs_plain"] == "200/200"
    assert 0 < s["continuous"]["gpu_busy_frac"] <= 1.0 and s["clocks"]["sm_mhz"] is not None
    assert set(s["continuous"]["by_field"]) == {"c128", "f64", "modp"}
