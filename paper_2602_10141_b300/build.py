"""Build libpermx.so (sm_103a) in-tree: nvcc for the CUDA sources, g++ for the
host sources, objects under _build/ at the repository root.

    python paper_2602_10141_b300/build.py [--force] [--jobs N]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libpermx.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]
CXX_FLAGS = ["-O2", "-fPIC", "-std=c++17", "-Wall", "-I" + INCLUDE, "-I" + CSRC,
             "-I" + os.path.join(CUDA_HOME, "include")]

# compile-time-n kernels are split into ranges so they build in parallel
INSTANCES = {
    "inst_modp.cu": [(1, 8), (9, 16), (17, 24), (25, 32), (33, 40), (41, 48)],
    "inst_f64.cu": [(1, 11), (12, 22), (23, 32)],
    "inst_c128.cu": [(1, 8), (9, 16), (17, 24), (25, 32)],
    "inst_x64r.cu": [(1, 11), (12, 22), (23, 32)],
    "inst_x64c.cu": [(1, 8), (9, 16), (17, 24), (25, 32)],
}
PLAIN_CU = ["batch.cu", "dispatch.cu", "peaks.cu", "noalloc.cu", "plan.cu", "stats.cu", "gather.cu", "selftest_dev.cu"]
PLAIN_CPP = ["api.cpp", "field.cpp", "schur.cpp", "serve.cpp", "selftest.cpp"]


def _gen_dispatch() -> None:
    """Write dispatch.cu and inst_range.inc (runtime n -> compile-time n)."""
    lines = ["// Expands PERMX_INST(N) for every N in [PERMX_NLO, PERMX_NHI] (N <= 48)."]
    for n in range(1, 49):
        lines.append(f"#if PERMX_NLO <= {n} && {n} <= PERMX_NHI\nPERMX_INST({n})\n#endif")
    _write_if_changed(os.path.join(CSRC, "inst_range.inc"), "\n".join(lines) + "\n")
    out = ["// Runtime-n dispatch to the compile-time-n kernels (written by build.py).",
           '#include "common.cuh"', "", "namespace permx {", ""]
    for kind, lt, mx in (("modp", "ModpLaunch", 48), ("f64", "FpLaunch", 32), ("c128", "FpLaunch", 32),
                         ("x64r", "FpLaunch", 32), ("x64c", "FpLaunch", 32)):
        out += [f"cudaError_t dispatch_{kind}(int n, const {lt}& L, cudaStream_t s) {{",
                "    const uint64_t items = L.item_end - L.item_begin;",
                "    if (items == 0) return cudaSuccess;",
                "    // blocks of kRyserThreads threads while the launch fills every SM; a",
                "    // smaller launch takes smaller blocks (down to one warp) so that its",
                "    // warps spread over more SMs instead of sharing a few (the results do",
                "    // not depend on the block size)",
                "    int threads = kRyserThreads;",
                "    auto grid_for = [&](int bps, int lanes_per_item = 1) {",
                "        const uint64_t lanes = items * lanes_per_item;",
                "        const uint64_t sms = (uint64_t)sm_count();",
                "        while (threads > 32 && (lanes + threads - 1) / threads < sms) threads >>= 1;",
                "        uint64_t want = (lanes + threads - 1) / threads;",
                "        uint64_t cap = sms * (uint64_t)bps * (uint64_t)(kRyserThreads / threads);",
                "        return (int)(want < cap ? want : cap);",
                "    };",
                "    switch (n) {"]
        for n in range(1, mx + 1):
            lanes = f"x64c_paired({n}) ? 2 : 1" if kind == "x64c" else "1"
            out.append(f"        case {n}: {{ const int g = grid_for(blocks_per_sm_{kind}<{n}>(), {lanes}); "
                       f"return launch_{kind}<{n}>(L, g, threads, s); }}")
        out += ["        default: return cudaErrorInvalidValue;", "    }", "}", ""]
    # resident blocks per SM of the kernel that a (kind, n) launch uses
    out += ["int dispatch_blocks_per_sm(int kind, int n) {",
            "    // kind: 0 modp, 1 f64, 2 c128, 3 x64 real, 4 x64 complex",
            "    switch (kind) {"]
    for k, (kind, mx) in enumerate((("modp", 48), ("f64", 32), ("c128", 32), ("x64r", 32), ("x64c", 32))):
        out.append(f"        case {k}:")
        out.append("            switch (n) {")
        for n in range(1, mx + 1):
            out.append(f"                case {n}: return blocks_per_sm_{kind}<{n}>();")
        out.append("                default: return 1;")
        out.append("            }")
    out += ["        default: return 1;", "    }", "}", ""]
    out.append("}  // namespace permx")
    _write_if_changed(os.path.join(CSRC, "dispatch.cu"), "\n".join(out) + "\n")


def _write_if_changed(path: str, text: str) -> None:
    if os.path.exists(path) and open(path).read() == text:
        return
    with open(path, "w") as f:
        f.write(text)


def _deps_hash(src: str, extra: list[str]) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cuh", ".h", ".inc")):
            h.update(open(os.path.join(CSRC, name), "rb").read())
    for name in sorted(os.listdir(INCLUDE)):
        h.update(open(os.path.join(INCLUDE, name), "rb").read())
    h.update(open(src, "rb").read())
    h.update(" ".join(extra).encode())
    return h.hexdigest()[:16]


def _jobs() -> list[tuple[str, list[str], str]]:
    jobs = []
    for src, ranges in INSTANCES.items():
        for lo, hi in ranges:
            obj = os.path.join(BUILD, f"{src[:-3]}_{lo}_{hi}.o")
            cmd = [NVCC] + NVCC_FLAGS + [f"-DPERMX_NLO={lo}", f"-DPERMX_NHI={hi}", "-c",
                                         os.path.join(CSRC, src), "-o", obj]
            jobs.append((os.path.join(CSRC, src), cmd, obj))
    for src in PLAIN_CU:
        obj = os.path.join(BUILD, src[:-3] + ".o")
        jobs.append((os.path.join(CSRC, src), [NVCC] + NVCC_FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj], obj))
    for src in PLAIN_CPP:
        obj = os.path.join(BUILD, src[:-4] + ".o")
        jobs.append((os.path.join(CSRC, src), ["g++"] + CXX_FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj], obj))
    return jobs


def _compile(job, force: bool) -> str:
    src, cmd, obj = job
    stamp = obj + ".stamp"
    key = _deps_hash(src, cmd)
    if not force and os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == key:
        return obj
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    with open(stamp, "w") as f:
        f.write(key)
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    _gen_dispatch()
    todo = _jobs()
    jobs = jobs or min(len(todo), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda j: _compile(j, force), todo))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + ".tmp"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


def ptxas_report(src: str = "inst_modp.cu", lo: int = 33, hi: int = 33) -> str:
    """Registers / spills / shared memory of one instantiation (-Xptxas -v)."""
    cmd = [NVCC] + NVCC_FLAGS + ["-Xptxas", "-v", f"-DPERMX_NLO={lo}", f"-DPERMX_NHI={hi}", "-c",
                                 os.path.join(CSRC, src), "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.stderr


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--clean", action="store_true")
    a = ap.parse_args()
    if a.clean and os.path.isdir(BUILD):
        shutil.rmtree(BUILD)
    build(force=a.force, jobs=a.jobs, verbose=True)
    sys.exit(0)
