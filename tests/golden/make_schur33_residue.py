"""Writes schur33_residue.txt: perm(S_33) mod p for the largest prime
p = 1 (mod 33) below 2^31, the first of the five primes of the exact-perm(S_33)
benchmark, computed by the oracle alone (plain Ryser mod p over all 2^33
subsets in binary order, row sums recomputed for every subset; paper §2.1).
About 50 minutes on 8 host cores.  Run from the repository root:
    python tests/golden/make_schur33_residue.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402


def main():
    n = 33
    p = O.primes_1_mod_n(n, 1)[0]
    g = O.primitive_nth_root(p, n)
    t = time.time()
    r = O.perm_modp(O.schur_residue_matrix(n, p, g), p)
    lines = ["# perm(S_33) mod p from the oracle (plain Ryser mod p over all 2^33 subsets, row sums",
             "# recomputed per subset; paper §2.1).  Written by make_schur33_residue.py",
             f"# in {time.time() - t:.0f} s.  Columns: n, p, primitive root g used, perm(S_33) mod p.",
             f"{n} {p} {g} {r}"]
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "schur33_residue.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(lines[-1])


if __name__ == "__main__":
    main()
