"""Writes schur_crt_oracle.txt: exact perm(S_n) for n = 21..31 computed by the
oracle alone (plain Ryser mod p in binary subset order, row sums recomputed for
every subset, then Chinese remaindering in Python integers; paper §2.1 method),
with one extra prime as a check and the bound |perm(S_n)|^2 <= n^n asserted.
It calls nothing but the oracle.  Run from the repository root:
    python tests/golden/make_schur_crt.py            # every n (about 2 hours on 8 cores)
    python tests/golden/make_schur_crt.py 30 31      # only these n; the other rows are kept
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402


NS = range(21, 32)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schur_crt_oracle.txt")


def main():
    header = ["# Exact perm(S_n) from the oracle: plain Ryser mod p (binary subset order) for the",
              "# largest primes p = 1 (mod n) below 2^31, Chinese remaindering in Python integers,",
              "# one more prime as a check (paper §2.1 method).  Written by make_schur_crt.py.",
              "# Columns: n, perm(S_n), primes used (the last one is the check prime)."]
    todo = [int(a) for a in sys.argv[1:]] or list(NS)
    assert all(n in NS for n in todo), todo
    rows = {}
    if sys.argv[1:] and os.path.exists(OUT):
        for ln in open(OUT):
            if ln.strip() and not ln.startswith("#"):
                rows[int(ln.split()[0])] = ln.rstrip("\n")
    for n in todo:
        k = O.prime_count_for(n)
        primes = O.primes_1_mod_n(n, k + 1)
        res = []
        for p in primes:
            S = O.schur_residue_matrix(n, p, O.primitive_nth_root(p, n))
            res.append(O.perm_modp(S, p))
        assert O.crt_modulus_suffices(n, primes[:k])
        value = O.crt(res[:k], primes[:k])
        assert value % primes[k] == res[k], n
        assert value * value <= n ** n, n
        rows[n] = f"{n} {value} " + " ".join(str(p) for p in primes)
        print(rows[n], flush=True)
        with open(OUT, "w") as f:        # after every n, so a long run keeps what it finished
            f.write("\n".join(header + [rows[m] for m in sorted(rows)]) + "\n")


if __name__ == "__main__":
    main()
