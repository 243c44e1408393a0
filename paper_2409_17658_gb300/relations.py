"""Relation records kept in a JSON file: checkpoint and resume of the per-m results.

For the transfer matrix A(G) of P_m, the first repeat A^(k+p) = q (x) A^k (Lemma 2) and
gamma(n) = min diag(A^n) for n = 1..k+p (Corollary 6) give gamma_R(P_m box C_n) for every n
(Prop. 7).  The library keeps one such record per m (include/rd.h, rd_relation_t); this module
writes records to a file and reads them back, so a later process, or a restarted query server,
answers those m without running their period searches again:

    {"format": "rd-relation-1", "records": [
        {"m": 9, "found": true, "k": 22, "p": 5, "q": 20, "j": 27, "gamma": [6, 10, 14, ...]}, ...]}

`gamma` lists gamma(1)..gamma(j).  Installing a record checks it against what every record of a
transfer matrix satisfies (rd_gamma_R_import); a wrong record that passes those checks gives wrong
answers, so load only files whose origin you trust.
"""
from __future__ import annotations

import json

from . import gamma_R_export, gamma_R_import

FORMAT = "rd-relation-1"
_KEYS = ("m", "found", "k", "p", "q", "j", "gamma")


def save(path: str, records: list[dict]) -> dict:
    """Write records (dicts as gamma_R_export / Server.export_relation return them); returns the document."""
    doc = {"format": FORMAT, "records": [{k: r[k] for k in _KEYS} for r in records]}
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    return doc


def load(path: str) -> list[dict]:
    """The records of a file written by save()."""
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != FORMAT:
        raise ValueError(f"{path}: not a relation file ({doc.get('format')!r})")
    recs = doc["records"]
    for r in recs:
        missing = [k for k in _KEYS if k not in r]
        if missing:
            raise ValueError(f"{path}: record without {missing}")
    return recs


def save_cache(path: str, ms) -> dict:
    """Export rd_gamma_R's records for the given m (searching those not cached yet) and save them."""
    return save(path, [gamma_R_export(m) for m in ms])


def load_cache(path: str) -> int:
    """Install every record of a file as rd_gamma_R's cache entry; returns how many."""
    recs = load(path)
    for r in recs:
        gamma_R_import(r)
    return len(recs)
