"""Relation records (checkpoint / resume of the per-m results), on the host.

A record -- the first repeat A^(k+p) = q (x) A^k (Lemma 2) and gamma(n) = min diag A^n for
n <= k + p (Corollary 6) -- fixes gamma_R(P_m box C_n) for every n (Prop. 7).  Records built by the
oracle are installed with rd_gamma_R_import; rd_gamma_R must then answer from them with no device
work (this file runs without a GPU, so any CUDA call would fail), and its answers are checked
against values that do not come from the record: the oracle's straight powering (Algorithm 1),
ceil(2n/3) for m = 1, and Remark 13's 2(m+1)n/5 for m >= 4 and 5 | n.
"""
import math

import pytest

from conftest import oracle_first_repeat


@pytest.fixture(scope="module")
def rd():
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    return rd


@pytest.fixture(autouse=True)
def clean_cache(rd):
    """Leave no imported record behind for later tests of rd_gamma_R."""
    rd.gamma_R_clear()
    yield
    rd.gamma_R_clear()


def oracle_record(orc, m, kmax=64):
    r = orc.power_until_periodic(m, kmax=kmax)
    assert r["found"]
    return dict(m=m, found=True, k=r["k"], p=r["p"], q=r["q"], j=r["j"], gamma=[int(v) for v in r["gamma"][1:]])


def golden_record(m):
    o = oracle_first_repeat(m)
    return dict(m=m, found=True, k=o["k"], p=o["p"], q=o["q"], j=o["j"], gamma=o["gamma"][1: o["j"] + 1])


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_import_answers_without_a_search(rd, orc, m):
    rd.gamma_R_import(oracle_record(orc, m))
    direct = orc.gamma_direct(m, 60)  # Algorithm 1, straight powering in the oracle
    for n in range(3, 61):
        assert rd.gamma_R(m, n) == direct[n], n
    for n in range(3, 3001):
        got = rd.gamma_R(m, n)
        if m == 1:
            assert got == math.ceil(2 * n / 3), n
        if m >= 4 and n % 5 == 0:
            assert got == 2 * (m + 1) * n // 5, n  # Remark 13


@pytest.mark.parametrize("m", [9, 10])
def test_import_of_the_oracles_stored_first_repeats(rd, m):
    """The oracle's row-streamed m = 9 and 10 results (golden files) answer every n on the host; beyond
    the stored powers, Remark 13 (5 | n) and the m = 9 closed form printed in Sec. 4.C check them."""
    rec = golden_record(m)
    rd.gamma_R_import(rec)
    for n in range(3, rec["j"] + 1):
        assert rd.gamma_R(m, n) == rec["gamma"][n - 1], n
    for n in range(3, 2001):
        got = rd.gamma_R(m, n)
        if n % 5 == 0:
            assert got == 2 * (m + 1) * n // 5, n
        if m == 9:
            assert got == (4 * n if n % 5 == 0 else 4 * n + 2), n


def test_export_returns_the_imported_record(rd, orc):
    rec = oracle_record(orc, 4)
    rd.gamma_R_import(rec)
    assert rd.gamma_R_export(4) == rec


def test_not_found_record(rd, orc):
    """A record without a relation answers n <= j and reports RD_NOT_FOUND beyond."""
    full = oracle_record(orc, 3)
    j = full["k"] + full["p"] - 1  # stop one power before the repeat
    rec = dict(m=3, found=False, k=None, p=None, q=None, j=j, gamma=full["gamma"][:j])
    rd.gamma_R_import(rec)
    assert rd.gamma_R_export(3) == rec
    for n in range(3, j + 1):
        assert rd.gamma_R(3, n) == full["gamma"][n - 1]
    with pytest.raises(rd.RdError) as e:
        rd.gamma_R(3, j + 1)
    assert e.value.status == rd.RD_NOT_FOUND


def _mutations(rec):
    """(name, record) pairs that break one rule rd_gamma_R_import checks."""
    out = []

    def mut(name, **kw):
        r = dict(rec, gamma=list(rec["gamma"]))
        r.update(kw)
        out.append((name, r))

    g = rec["gamma"]
    mut("m zero", m=0)
    mut("m too large", m=16)
    mut("p zero", p=0, j=rec["k"], gamma=g[: rec["k"]])
    mut("k zero", k=0, p=rec["k"] + rec["p"])
    mut("q inconsistent", q=rec["q"] + 1)
    mut("negative gamma", gamma=[-1] + g[1:])
    mut("gamma above 2mn", gamma=g[:2] + [2 * rec["m"] * 3 + 1] + g[3:])
    mut("found zero with a period", found=False)
    return out


def test_import_rejects_inconsistent_records(rd, orc):
    good = oracle_record(orc, 5)
    rd.gamma_R_import(good)
    for name, bad in _mutations(good):
        if name == "found zero with a period":
            # the binding drops k, p, q when found is false; send the fields as given instead
            rel, gamma = rd._relation_args(dict(bad, found=True))
            rel.found = 0
            st = rd._lib().rd_gamma_R_import(rd.ctypes.byref(rel), gamma.ctypes.data)
            assert st == rd.RD_ERR_ARG, name
            continue
        m_ok = 1 <= bad["m"] <= rd.RD_MAX_M
        with pytest.raises(rd.RdError) as e:
            rd.gamma_R_import(bad)
        assert e.value.status == rd.RD_ERR_ARG, name
        if m_ok:
            assert rd.gamma_R_export(bad["m"]) == good, name  # the cache entry is unchanged
    # null pointers and a record whose j disagrees with its gamma list
    assert rd._lib().rd_gamma_R_import(None, None) == rd.RD_ERR_ARG
    with pytest.raises(ValueError):
        rd._relation_args(dict(good, j=good["j"] + 1))


def test_export_rejects_short_gamma_buffer(rd, orc):
    rec = oracle_record(orc, 2)
    rd.gamma_R_import(rec)
    rel = rd.Relation()
    buf = (rd.ctypes.c_int64 * rec["j"])()  # one entry short of j + 1
    assert rd._lib().rd_gamma_R_export(2, rd.ctypes.byref(rel), buf, rec["j"]) == rd.RD_ERR_ARG
    assert rel.j == rec["j"] and rel.k == rec["k"] and rel.p == rec["p"] and rel.q == rec["q"]
    assert rd._lib().rd_gamma_R_export(0, rd.ctypes.byref(rel), None, 0) == rd.RD_ERR_ARG


def test_relation_file_round_trip(rd, orc, tmp_path):
    from paper_2409_17658_gb300 import relations

    recs = [oracle_record(orc, m) for m in (1, 2, 3)] + [golden_record(9)]
    for r in recs:
        rd.gamma_R_import(r)
    path = str(tmp_path / "relations.json")
    relations.save_cache(path, [1, 2, 3, 9])
    before = {(m, n): rd.gamma_R(m, n) for m in (1, 2, 3, 9) for n in range(3, 400)}
    rd.gamma_R_clear()
    assert relations.load_cache(path) == 4
    assert relations.load(path) == recs
    after = {(m, n): rd.gamma_R(m, n) for m in (1, 2, 3, 9) for n in range(3, 400)}
    assert after == before
    bad = tmp_path / "other.json"
    bad.write_text('{"format": "rd-tune-1", "entries": []}')
    with pytest.raises(ValueError):
        relations.load(str(bad))


def test_command_line_answers_from_a_relation_file(rd, tmp_path):
    """python -m paper_2409_17658_gb300 gamma M N --relations FILE answers on the host from the saved record
    (no GPU here); m = 9 against the closed form printed in Sec. 4.C."""
    import json
    import os
    import subprocess
    import sys

    from paper_2409_17658_gb300 import relations

    path = str(tmp_path / "rel.json")
    relations.save(path, [golden_record(9)])
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ns = [3, 7, 27, 28, 500, 12345]
    out = subprocess.run([sys.executable, "-m", "paper_2409_17658_gb300", "gamma", "9", *map(str, ns), "--relations",
                          path], cwd=root, capture_output=True, text=True, check=True).stdout
    got = [json.loads(line)["gamma_R"] for line in out.splitlines()]
    assert got == [4 * n if n % 5 == 0 else 4 * n + 2 for n in ns]
