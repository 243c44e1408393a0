"""Writes oracle_m<M>_first_repeat.txt: the oracle's first repeat and gamma values for one m.

For m = 9 (N = 21909) and m = 10 (N = 64769) the oracle's dense search would hold about 27 powers
of 3.8 GB or 30 of 34 GB, so this uses its row-streamed form (Algorithm 2 with the first-repeat rule,
one start word at a time).  It calls only the oracle.  Run from the repository root:

    python tests/golden/make_oracle_first_repeat.py 9 30     # about 5 minutes on 8 cores
    python tests/golden/make_oracle_first_repeat.py 10 31    # about 80 minutes on 8 cores
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

TABLE2 = {9: "Table 2 prints (n0, alpha, beta) = (22, 5, 20) for m = 9.",
          10: "Table 2 stops at m = 9; Cor. 12 gives gamma = 22 n / 5 for n = 0 mod 5, n >= 10."}


def main(m: int, kmax: int) -> None:
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_m{m}_first_repeat.txt")
    t0 = time.time()
    r = oracle.power_until_periodic_rows(m, kmax=kmax)
    dt = time.time() - t0
    assert r["found"], "no repeat up to kmax"
    with open(out, "w") as fh:
        fh.write(f"# m = {m}: the oracle's first repeat A^(k+p) = q (x) A^k and gamma[n] = min diag A^n, n = 1..{kmax}\n")
        fh.write("# (Algorithm 2 with the first-repeat rule, Corollary 6).  Written by make_oracle_first_repeat.py, which\n")
        fh.write(f"# calls oracle.power_until_periodic_rows({m}, kmax={kmax}) only ({oracle.threads()} threads, {dt:.0f} s).\n")
        fh.write(f"# {TABLE2.get(m, '')}\n")
        fh.write("# m k p q j\n")
        fh.write(f"{m} {r['k']} {r['p']} {r['q']} {r['j']}\n")
        fh.write("# n gamma\n")
        for n in range(1, kmax + 1):
            fh.write(f"{n} {int(r['gamma'][n])}\n")
    print(f"wrote {out}: (k,p,q,j) = ({r['k']},{r['p']},{r['q']},{r['j']}) in {dt:.0f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]), int(sys.argv[2]))
