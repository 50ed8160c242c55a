"""bench.py's reference arm on the CPU (it runs only the oracle): one JSON
line with the keys the bench contract asks for, and under a multi-rank
launch only rank 0 prints it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, extra_args=()):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", *extra_args], capture_output=True, text=True, timeout=300, env=env,
                       cwd=ROOT)
    return r


def test_reference_arm_json_line():
    r = _run({"OMP_NUM_THREADS": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "ryser_terms_per_s" and d["unit"] == "terms/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["config"]["workload"] == "schur_n33_fp_5primes" and len(d["config"]["prime_list"]) == 5
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == 2 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_are_silent():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2", "OMP_NUM_THREADS": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_jsonl_log_copies_the_result_line(tmp_path):
    """--jsonl appends each printed JSON line, stamped with the time and the
    arguments, and leaves stdout unchanged."""
    log = tmp_path / "runs.jsonl"
    for _ in range(2):
        r = _run({"OMP_NUM_THREADS": "1"}, ("--jsonl", str(log)))
        assert r.returncode == 0, r.stderr[-2000:]
    printed = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    logged = [json.loads(ln) for ln in log.read_text().splitlines()]
    assert len(printed) == 1 and len(logged) == 2
    for rec in logged:
        assert rec["impl"] == "reference" and rec["metric"] == printed[0]["metric"]
        assert rec["logged_at"] and "--jsonl" in rec["argv"]
    assert "logged_at" not in printed[0]


def test_cpu_baseline_on_the_host():
    """bench.py's cpu_baseline leg runs on the CPU alone: the oracle on all
    cores and on one, and the plain Gray walk on one thread and on all."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    n = 33
    primes = O.primes_1_mod_n(n, 1)
    mats = [O.schur_residue_matrix(n, p, O.primitive_nth_root(p, n)) for p in primes]
    cb = bench.cpu_baseline(primes, mats, target_s=0.4)
    assert cb["kind"] == "oracle" and cb["unit"] == "terms/s" and cb["value"] > 0 and cb["cores"] >= 1
    for key in ("single_core", "gray_walk_single_core", "gray_walk_all_cores"):
        assert cb[key]["value"] > 0 and cb[key]["cores"] >= 1 and cb[key]["sample"], key
    assert cb["gray_walk_all_cores"]["cores"] == cb["cores"]
