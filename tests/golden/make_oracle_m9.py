"""Writes oracle_m9_first_repeat.txt: the oracle's first repeat and gamma values for m = 9.

The oracle's dense search would hold 27 powers of 3.8 GB each at m = 9 (N = 21909), so this uses
its row-streamed form (Algorithm 2 with the first-repeat rule, one start word at a time).  It calls
only the oracle.  Run from the repository root:  python tests/golden/make_oracle_m9.py
(about 5 minutes on 8 cores).
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

M, KMAX = 9, 30
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_m9_first_repeat.txt")


def main() -> None:
    t0 = time.time()
    r = oracle.power_until_periodic_rows(M, kmax=KMAX)
    dt = time.time() - t0
    assert r["found"], "no repeat up to kmax"
    with open(OUT, "w") as fh:
        fh.write(f"# m = {M}: the oracle's first repeat A^(k+p) = q (x) A^k and gamma[n] = min diag A^n, n = 1..{KMAX}\n")
        fh.write("# (Algorithm 2 with the first-repeat rule, Corollary 6).  Written by make_oracle_m9.py, which\n")
        fh.write(f"# calls oracle.power_until_periodic_rows({M}, kmax={KMAX}) only ({oracle.threads()} threads, {dt:.0f} s).\n")
        fh.write("# Table 2 prints (n0, alpha, beta) = (22, 5, 20) for m = 9.\n")
        fh.write("# m k p q j\n")
        fh.write(f"{M} {r['k']} {r['p']} {r['q']} {r['j']}\n")
        fh.write("# n gamma\n")
        for n in range(1, KMAX + 1):
            fh.write(f"{n} {int(r['gamma'][n])}\n")
    print(f"wrote {OUT}: (k,p,q,j) = ({r['k']},{r['p']},{r['q']},{r['j']}) in {dt:.0f} s")


if __name__ == "__main__":
    main()
