"""The oracle and the CUDA path share no code: no import, include or link in
either direction, and nothing committed reads the working folder.  Checked on
the source text (CPU only)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2602_10141_b300")
ORACLE = os.path.join(ROOT, "oracle")
SRC_EXT = (".py", ".c", ".cu", ".cuh", ".cpp", ".h", ".inc")


def _files(top):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build", "obj")]
        for f in files:
            if f.endswith(SRC_EXT):
                yield os.path.join(d, f)


def _code_lines(path):
    """Source lines with comments and docstrings left in: the patterns below
    only match import / include statements, which comments do not form."""
    with open(path, encoding="utf-8", errors="replace") as fh:
        return fh.read().splitlines()


def test_product_never_imports_or_includes_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b|from\s+\.\.?oracle\b|#\s*include\s*[<\"].*oracle)")
    bad = [(p, ln) for p in _files(PKG) for ln in _code_lines(p) if pat.search(ln)]
    bad += [(p, ln) for p in _files(os.path.join(ROOT, "include")) for ln in _code_lines(p) if pat.search(ln)]
    assert not bad, bad


def test_oracle_never_imports_or_includes_the_product():
    pat = re.compile(r"^\s*(import\s+paper_2602_10141_b300\b|from\s+paper_2602_10141_b300\b|"
                     r"#\s*include\s*[<\"](permx|.*csrc/|common\.cuh|x64_arith|ryser_))")
    bad = [(p, ln) for p in _files(ORACLE) for ln in _code_lines(p) if pat.search(ln)]
    assert not bad, bad


def test_product_loads_no_oracle_library():
    for p in _files(PKG):
        for ln in _code_lines(p):
            assert "liboracle" not in ln and "libcpuwalk" not in ln, (p, ln)


def test_nothing_committed_reads_the_working_folder():
    tops = [PKG, ORACLE, os.path.join(ROOT, "tests"), os.path.join(ROOT, "workloads"), os.path.join(ROOT, "include")]
    files = [f for t in tops for f in _files(t)]
    files += [os.path.join(ROOT, f) for f in ("bench.py", "bench_workloads.py", "__graft_entry__.py")]
    me = os.path.abspath(__file__)
    for p in files:
        if os.path.abspath(p) == me:
            continue
        for ln in _code_lines(p):
            assert "_work/" not in ln and "_work\\\\" not in ln and "'_work'" not in ln and '"_work"' not in ln, (p, ln)


def test_package_refuses_to_import_without_its_library(tmp_path):
    """No fallback: a copy of the package without libpermx.so fails to import."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2602_10141_b300"
    pkg.mkdir()
    shutil.copy(os.path.join(PKG, "__init__.py"), pkg / "__init__.py")
    r = subprocess.run([sys.executable, "-c", "import paper_2602_10141_b300"], cwd=str(tmp_path),
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "is missing" in r.stderr
