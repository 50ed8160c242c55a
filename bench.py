"""Benchmark: exact perm(S_33) over F_p, 5 primes just below 2^31 (the
Schur-matrix workload of paper §2.1), Gray-code Ryser terms per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step is one pass of the whole hot path over the workload: the 5 residue
matrices (g^{jk} mod p), resident in HBM, go through chunk planning, the
Gray-code walk, the reductions and the finalisation in one batched
``perm_modp`` call; the host CRT of the 5 residues closes the step.  `value`
counts Ryser terms the way the formula states them, n * 2^n per permanent
(5 * 33 * 2^33 per step), divided by the device time (CUDA events on the
launching stream), summed over ranks.  The kernels evaluate the
Nijenhuis-Wilf form of the same formula, which needs n * 2^(n-1) terms per
permanent; `terms_evaluated_per_s` and the roofline use that actual count.  ``e2e`` repeats the measurement
through the host-buffer call ``perm_modp_host`` (copies inside the timed
region).  With N > 1 (torchrun) every rank computes its own, disjoint set of
5 primes (weak scaling, no collective on the data path).

``--impl reference`` times the CPU oracle (the plain Ryser evaluation, row
sums recomputed for every subset, OpenMP over the machine's cores) on a bounded
sample of the same workload and reports the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 33
NPRIMES = 5
METRIC = "ryser_terms_per_s"
UNIT = "terms/s"
WORKLOAD = "schur_n33_fp_5primes"
# dram__bytes_read.sum + dram__bytes_write.sum of one ryser_modp_kernel<33> launch of the
# small case (bench.py --profile-case: 2^30 Gray steps of S_33 mod p, the same kernel), from
# one ncu capture of the current build; not scaled to the bench launch (5 x 2^32 steps): the
# walk reads its residue tables once and otherwise only instruction fetch reaches DRAM, which
# does not grow in proportion to the launch
WALK_DRAM_BYTES_SMALL_CASE = 37_632


def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_prime_skip(rank: int) -> int:
    """Rank r of a weak-scaling run takes primes [5r, 5r + 5) of the descending
    list of primes p = 1 (mod 33) below 2^31: disjoint sets, each enough for
    the CRT bound, so every rank reconstructs perm(S_33) independently."""
    return NPRIMES * rank


def field_setup(n: int, count: int, skip: int):
    """Primes, roots and residue matrices through the library's host helpers."""
    import paper_2602_10141_b300 as px
    primes = px.perm_primes_1_mod_n(n, count, skip)
    mats = [px.perm_schur_residues(n, p, px.perm_primitive_root(p, n)) for p in primes]
    return primes, mats


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def device_info(torch, index: int) -> dict:
    """The GPU and host the numbers were taken on."""
    prop = torch.cuda.get_device_properties(index)
    return {"name": prop.name, "sm_count": prop.multi_processor_count,
            "memory_gib": round(prop.total_memory / 2 ** 30, 1), "host_cores": os.cpu_count()}


class _JsonlTee:
    """Copies every JSON object line written to stdout into a JSONL log, with
    the time it was written (``--jsonl PATH``)."""

    def __init__(self, stream, path: str):
        self.stream, self.path, self.buf = stream, path, ""

    def write(self, text: str) -> int:
        self.buf += text
        while "\n" in self.buf:
            line, self.buf = self.buf.split("\n", 1)
            if line.startswith("{"):
                try:
                    rec = json.loads(line)
                except ValueError:
                    rec = None
                if isinstance(rec, dict):
                    rec.setdefault("logged_at", time.strftime("%Y-%m-%dT%H:%M:%S%z"))
                    rec.setdefault("argv", sys.argv[1:])
                    with open(self.path, "a") as f:
                        f.write(json.dumps(rec) + "\n")
        return self.stream.write(text)

    def flush(self):
        self.stream.flush()

    def __getattr__(self, name):
        return getattr(self.stream, name)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(primes, mats, target_s: float = 16.0):
    """The oracle's Ryser evaluation (row sums recomputed for every subset) on a
    bounded Gray-index range of the first prime's matrix, timed on the host."""
    import oracle as O
    A, p = mats[0], primes[0]
    k0 = 1 << 31
    O.ryser_modp_gray_range(A, p, k0, k0 + (1 << 12))   # start the OpenMP threads
    span = 1 << 23                       # ~1 s on 16 cores: long enough for a stable rate
    t0 = time.perf_counter()
    O.ryser_modp_gray_range(A, p, k0, k0 + span)
    dt = time.perf_counter() - t0
    rate = span / max(dt, 1e-9)
    span = int(min(max(rate * target_s, 1 << 16), 1 << 30))
    t0 = time.perf_counter()
    O.ryser_modp_gray_range(A, p, k0, k0 + span)
    dt = time.perf_counter() - t0
    cores = O.num_threads()
    # the same oracle on one core, on a sample 1/cores as long (about the same seconds)
    O.set_num_threads(1)
    span1 = max(span // max(cores, 1), 1 << 16)
    t1 = time.perf_counter()
    O.ryser_modp_gray_range(A, p, k0, k0 + span1)
    dt1 = time.perf_counter() - t1
    O.set_num_threads(cores)
    # the paper's own CPU algorithm (incremental Gray walk), the comparator for
    # its GPU-over-CPU speed-ups: on one thread (its single-threaded figure)
    # and with one Gray block per host core (its multi-core figure), each for
    # about target_s / 4 seconds
    from oracle import cpu_walk as W
    walk_s = target_s / 4
    W.modp_gray_range(A, p, k0, k0 + (1 << 14))
    t2 = time.perf_counter()
    W.modp_gray_range(A, p, k0, k0 + (1 << 16))
    rate_w = (1 << 16) / max(time.perf_counter() - t2, 1e-9)
    span_w = int(min(max(rate_w * walk_s, 1 << 16), 1 << 30))
    t2 = time.perf_counter()
    W.modp_gray_range(A, p, k0, k0 + span_w)
    dt2 = time.perf_counter() - t2
    span_m = int(min(span_w * max(cores, 1), 1 << 31))
    t3 = time.perf_counter()
    _, threads_m = W.modp_gray_range_mt(A, p, k0, k0 + span_m)
    dt3 = time.perf_counter() - t3
    # the block split of the multi-core walk, checked against the oracle on a short range
    ka = k0 + (1 << 29) + 12345
    mt_ok = W.modp_gray_range_mt(A, p, ka, ka + (1 << 20) + 7)[0] == O.ryser_modp_gray_range(A, p, ka,
                                                                                             ka + (1 << 20) + 7)
    assert mt_ok, "multi-core CPU walk disagrees with the oracle"
    return {"value": N * span / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"Gray indices [{k0}, {k0 + span}) of S_33 mod {p} (one of 5 primes), "
                      f"{span} subsets x {N} rows, {dt:.1f} s",
            "single_core": {"value": N * span1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"Gray indices [{k0}, {k0 + span1}), {dt1:.1f} s"},
            "gray_walk_single_core": {"value": N * span_w / dt2, "unit": UNIT, "cores": 1,
                                      "kind": "plain CPU Gray-code walk (incremental row sums, uint64 %)",
                                      "sample": f"Gray indices [{k0}, {k0 + span_w}), {dt2:.1f} s"},
            "gray_walk_all_cores": {"value": N * span_m / dt3, "unit": UNIT, "cores": threads_m,
                                    "checked_against_oracle": f"Gray indices [{ka}, {ka + (1 << 20) + 7})",
                                    "kind": "the same walk, one contiguous Gray block per host thread",
                                    "sample": f"Gray indices [{k0}, {k0 + span_m}), {dt3:.1f} s"}}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle as O
    primes = O.primes_1_mod_n(N, NPRIMES)
    mats = [O.schur_residue_matrix(N, p, O.primitive_nth_root(p, N)) for p in primes]
    # calibrate a per-step sample of about 3 s
    k0 = 1 << 31
    O.ryser_modp_gray_range(mats[0], primes[0], k0, k0 + (1 << 12))   # start the OpenMP threads
    t0 = time.perf_counter()
    O.ryser_modp_gray_range(mats[0], primes[0], k0, k0 + (1 << 19))
    rate = (1 << 19) / max(time.perf_counter() - t0, 1e-9)
    span = int(min(max(rate * 3.0, 1 << 16), 1 << 30))
    for w in range(args.warmup):
        O.ryser_modp_gray_range(mats[w % NPRIMES], primes[w % NPRIMES], k0, k0 + (1 << 14))
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        O.ryser_modp_gray_range(mats[s % NPRIMES], primes[s % NPRIMES], k0, k0 + span)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = N * span * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N, "primes": NPRIMES, "prime_list": primes},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{span} Gray indices of S_33 per step (bounded sample; the full "
                                       f"step is {NPRIMES} x 2^33 subsets)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def multiply_pipe_bound(px, sms: int) -> dict:
    """Evaluated terms/s that the F_p walk's multiplies allow on this GPU now:
    a term needs one mul.wide, one mul.lo and one mul.hi (signed Montgomery
    product), all on the integer-multiply pipe, so the bound is
    1 / (1/R_wide + 1/R_lo + 1/R_hi) with each R the whole-GPU issue rate the
    library's probe kernels measure (8 independent chains per thread, 8
    blocks of 256 threads per SM)."""
    rates = {}
    for name, kind in (("mul_wide_u32", 5), ("mad_lo_u32", 4), ("mul_hi_u32", 6)):
        px.permx_peak_probe(kind, sms * 8, 256, 1024)            # warm-up
        ops, ms = px.permx_peak_probe(kind, sms * 8, 256, 8192)
        rates[name] = ops
    bound = 1.0 / sum(1.0 / r for r in rates.values())
    return {"bound_terms_per_s": bound, "rates_ops_per_s": rates}


def run_profile_case():
    import torch
    import paper_2602_10141_b300 as px
    primes, mats = field_setup(N, 1, 0)
    dA = torch.from_numpy(mats[0].astype(np.int32).reshape(-1)).cuda()
    for _ in range(3):
        r = px.perm_modp_gray_range(dA, N, primes[0], 0, 1 << 30)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "S_33 mod p, Gray indices [0, 2^30)", "p": primes[0], "residue": r}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for ncu: the same kernel over 2^30 Gray indices of S_33 mod one prime")
    ap.add_argument("--workload", default="schur33",
                    choices=["schur33", "haar14_plain", "ensembles_batched", "serving", "profile_fp", "schur_long",
                             "paper_tables", "profile_stats", "batch_scaling", "orthogonal_large",
                             "lognormal_large"],
                    help="schur33 is the headline; the others measure the plain, batched and served paths")
    ap.add_argument("--ns", default="", help="schur_long: comma-separated n (default 36..43)")
    ap.add_argument("--ckpt-dir", default="", help="schur_long: keep checkpoints here (resume from them)")
    ap.add_argument("--disjoint", action="store_true",
                    help="schur_long: use primes disjoint from the default set (a cross-check of a long run)")
    ap.add_argument("--max-slices", type=int, default=0,
                    help="schur_long: stop after this many checkpointed slices per n (0 = run to the end)")
    ap.add_argument("--scale", type=float, default=0.02,
                    help="ensembles_batched / serving: fraction of the full sample counts")
    ap.add_argument("--jsonl", default="",
                    help="also append every JSON result line (with a timestamp and the arguments) to this file")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the plain, batched and served measurements added to the line")
    ap.add_argument("--extras-scale", type=float, default=1.0,
                    help="fraction of the full sample counts for the batched and served measurements")
    args = ap.parse_args()
    rank, world, local = _rank_env()
    if args.jsonl and rank == 0:
        sys.stdout = _JsonlTee(sys.stdout, args.jsonl)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.profile_case:
        return run_profile_case()
    if args.workload != "schur33":
        import bench_workloads
        return bench_workloads.run(args)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2602_10141_b300 as px

    # every rank: its own 5 primes (disjoint sets), residue matrices resident in HBM
    primes, mats = field_setup(N, NPRIMES, skip=rank_prime_skip(rank))
    flat = np.concatenate([m.reshape(-1) for m in mats]).astype(np.uint32)
    n_arr = np.full(NPRIMES, N, np.int32)
    off = np.arange(NPRIMES, dtype=np.int64) * N * N
    dA = torch.from_numpy(flat.view(np.int32)).cuda()
    out = torch.empty(NPRIMES, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    units_per_step = NPRIMES * N * (1 << N)          # nominal Ryser terms
    evaluated_per_step = NPRIMES * N * (1 << (N - 1))  # terms the Nijenhuis-Wilf walk evaluates
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MiB > 126 MB L2

    def step():
        px.perm_modp(dA, n_arr, off, primes, out, stream)

    def crt_of(res):
        return px.perm_crt([int(x) & 0xFFFFFFFF for x in res], primes)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    value_ref = crt_of(out.cpu().numpy())
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    bound = multiply_pipe_bound(px, sms)

    # timed region: per-step CUDA events, L2 flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            step()
            ev[s][1].record(stream)
            res = out.cpu().numpy()          # D2H of the step's result (5 residues) and host CRT
            assert crt_of(res) == value_ref
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    if world > 1:
        dist.barrier()
    dev_s = sum(ms) / 1e3
    t_local = torch.tensor([dev_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    t_max = float(t_local.item())
    value = units_per_step * args.steps * world / t_max

    # end to end through the host-buffer call: copies in and out inside the timed region
    # inputs and results in pinned host memory (the copies inside perm_modp_host are DMA)
    host_flat = torch.from_numpy(flat.view(np.int32).copy()).pin_memory().numpy().view(np.uint32)
    e2e_out = torch.empty(NPRIMES, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    for _ in range(2):
        px.perm_modp_host(host_flat, n_arr, off, primes, e2e_out, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(args.steps):
        px.perm_modp_host(host_flat, n_arr, off, primes, e2e_out, stream)
        assert crt_of(e2e_out) == value_ref
    e2e_s = time.perf_counter() - t0
    t_e2e = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t_e2e, op=dist.ReduceOp.MAX)
    e2e_value = units_per_step * args.steps * world / float(t_e2e.item())

    extras = {}
    if world == 1 and not args.no_extras:
        # the batched, plain and served halves of the metric, each with its own clock record
        import bench_workloads as BW
        extras["plain"] = BW.plain_object()
        extras["batched"] = BW.batched_object(args.extras_scale)
        extras["served"] = BW.served_object(args.extras_scale)

    if rank == 0:
        # integer-issue roofline of the F_p walk: one term = 1 modular add + 1 Montgomery
        # multiply; the multiply pipe (mul.wide + mul.lo + mul.hi per term) binds, at the
        # rates the library's probes measured on this GPU just before the timed region
        cs = clk.summary()
        peak = bound["bound_terms_per_s"]
        achieved = evaluated_per_step / (statistics.median(ms) / 1e3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "primes": NPRIMES, "prime_sets": "disjoint per rank",
                       "l2": "flushed between steps (256 MiB write)", "units_per_step": units_per_step,
                       "form": "Nijenhuis-Wilf (2^(n-1) Gray steps per permanent)",
                       "perm_S33": str(value_ref)},
            "perms_per_s": NPRIMES * args.steps * world / t_max,
            "terms_evaluated_per_s": evaluated_per_step * args.steps * world / t_max,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tterms/s",
                         "frac": achieved / peak, "traffic": WALK_DRAM_BYTES_SMALL_CASE,
                         "traffic_unit": "bytes per launch of the 2^30-step small case of the same kernel "
                                         "(ncu, current build; residue tables + instruction fetch, not scaled)",
                         "kernel": f"ryser_modp_kernel<{N}>",
                         "peak_source": "integer-multiply-pipe bound 1/(1/R_wide + 1/R_lo + 1/R_hi) from the "
                                        "library's issue-rate probes run in this process (permx_peak_probe)",
                         "probe_rates_ops_per_s": bound["rates_ops_per_s"]},
            "clocks": cs,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(flat.nbytes),
                    "d2h_bytes_per_step": 4 * NPRIMES},
            "gpu_launches": 4 * args.steps,   # metadata, staging, Gray walk, finalize per step
            "device": device_info(torch, local),
        }
        line.update(extras)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(primes, mats)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
