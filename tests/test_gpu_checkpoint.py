"""Checkpointed exact perm(S_n) (paper §2.1 method over many slices): a run
stopped after some slices, or a process killed mid-run, resumes from its
checkpoint file to the same integer as an uninterrupted run; the failure is
made on the host (a slice limit, SIGKILL between slices), never on the GPU."""
import os
import signal
import subprocess
import sys
import time

import pytest

import oracle as O

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def px():
    import paper_2602_10141_b300 as px
    return px


def test_slice_limit_then_resume(px, tmp_path):
    n = 19
    ck = str(tmp_path / "s19.ckpt")
    with pytest.raises(px.PermxError) as e:
        px.perm_schur_crt_ex(n, 0, ck, slice_subsets=1 << 14, max_slices=7)
    assert e.value.code == px.PERMX_EAGAIN
    text = open(ck).read()
    assert text.startswith("permx-schur-ckpt 2") and "cursor" in text
    v, primes, res = px.perm_schur_crt_ex(n, 0, ck, slice_subsets=1 << 14)
    assert v == O.schur_exact(n)
    # a finished checkpoint answers again without recomputation
    assert px.perm_schur_crt_ex(n, 0, ck)[0] == v


def test_killed_process_resumes(px, tmp_path):
    n = 29
    ck = str(tmp_path / "s29.ckpt")
    code = ("import sys; sys.path.insert(0, %r); import paper_2602_10141_b300 as px; "
            "px.perm_schur_crt_ex(%d, 0, %r, slice_subsets=1 << 22)" % (ROOT, n, ck))
    proc = subprocess.Popen([sys.executable, "-c", code], start_new_session=True)
    t0 = time.time()
    while not os.path.exists(ck) and time.time() - t0 < 120 and proc.poll() is None:
        time.sleep(0.05)
    time.sleep(0.3)
    if proc.poll() is None:
        os.killpg(proc.pid, signal.SIGKILL)   # host-side failure between or during slices
    proc.wait()
    assert os.path.exists(ck)
    resumed = px.perm_schur_crt_ex(n, 0, ck, slice_subsets=1 << 22)[0]
    fresh = px.perm_schur_crt_ex(n, 0, None)[0]
    assert resumed == fresh
    assert fresh * fresh <= n ** n
    # disjoint prime sets agree (an independent check on the integer)
    other = O.primes_1_mod_n(n, 5, skip=6)
    import numpy as np
    import torch
    mats = [O.schur_residue_matrix(n, p, O.primitive_nth_root(p, n)) for p in other]
    flat = np.concatenate([m.reshape(-1) for m in mats]).astype(np.int32)
    out = torch.empty(5, dtype=torch.int32, device="cuda")
    px.perm_modp(torch.from_numpy(flat).cuda(), [n] * 5, [i * n * n for i in range(5)], other, out)
    assert O.crt([int(x) & 0xFFFFFFFF for x in out.cpu().numpy()], other) == fresh
