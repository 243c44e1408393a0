"""Command line: gamma_R(P_m box C_n) and the relation records behind it.

    python -m paper_2409_17658_gb300 gamma M N [N ...] [--relations FILE]
        gamma_R(P_M box C_N) for each N (Corollary 6; beyond the stored powers, Prop. 7 from the first
        repeat).  With --relations, records saved earlier are installed first, so no period search runs
        for the m they cover.
    python -m paper_2409_17658_gb300 relation M [M ...] [--save FILE]
        the first repeat A^(k+p) = q (x) A^k of each M (Lemma 2) and gamma(1..k+p), as JSON lines or saved
        to FILE (format of paper_2409_17658_gb300.relations).

The period search of an m not covered by a record runs on the current CUDA device.
"""
from __future__ import annotations

import argparse
import json
import sys

from . import gamma_R, gamma_R_export, relations


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2409_17658_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("gamma", help="gamma_R(P_m box C_n)")
    g.add_argument("m", type=int)
    g.add_argument("n", type=int, nargs="+")
    g.add_argument("--relations", default="", metavar="FILE", help="install saved relation records first")
    r = sub.add_parser("relation", help="the first repeat of A(G) and its gamma table")
    r.add_argument("m", type=int, nargs="+")
    r.add_argument("--save", default="", metavar="FILE", help="write the records to FILE instead of stdout")
    args = ap.parse_args(argv)
    if args.cmd == "gamma":
        if args.relations:
            relations.load_cache(args.relations)
        for n in args.n:
            print(json.dumps({"m": args.m, "n": n, "gamma_R": gamma_R(args.m, n)}))
        return 0
    recs = [gamma_R_export(m) for m in args.m]
    if args.save:
        relations.save(args.save, recs)
    else:
        for rec in recs:
            print(json.dumps(rec))
    return 0


if __name__ == "__main__":
    sys.exit(main())
