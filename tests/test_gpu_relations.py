"""Relation records on a GB300: what the GPU search records equals the oracle's first repeat, and a query
server warm-started from records answers every query on the host, without a single period search."""
import pytest

from conftest import oracle_first_repeat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    rd.gamma_R_clear()
    yield rd
    rd.gamma_R_clear()


def oracle_record(orc, m, kmax=64):
    r = orc.power_until_periodic(m, kmax=kmax)
    assert r["found"]
    return dict(m=m, found=True, k=r["k"], p=r["p"], q=r["q"], j=r["j"], gamma=[int(v) for v in r["gamma"][1:]])


def golden_record(m):
    o = oracle_first_repeat(m)
    return dict(m=m, found=True, k=o["k"], p=o["p"], q=o["q"], j=o["j"], gamma=o["gamma"][1: o["j"] + 1])


def closed_form(rec, n):
    """Prop. 7 from a record's boundary values."""
    if n <= rec["j"]:
        return rec["gamma"][n - 1]
    k, p = rec["k"], rec["p"]
    return rec["gamma"][k + (n - k) % p - 1] + rec["q"] * ((n - k) // p)


def test_export_after_the_gpu_search_equals_the_oracle(rd, orc):
    """rd_gamma_R_export runs the GPU search (single-CTA for m <= 4, row split from m = 5) and records
    exactly the oracle's first repeat and gamma table; after a clear, importing that record reproduces
    every answer."""
    rd.gamma_R_clear()
    recs = {}
    for m in range(1, 8):
        recs[m] = rd.gamma_R_export(m)
        assert recs[m] == oracle_record(orc, m), m
    answers = {(m, n): rd.gamma_R(m, n) for m in recs for n in range(3, 300)}
    rd.gamma_R_clear()
    for r in recs.values():
        rd.gamma_R_import(r)
    assert {(m, n): rd.gamma_R(m, n) for m in recs for n in range(3, 300)} == answers
    rd.gamma_R_clear()


def test_server_warm_start_runs_no_search(rd, orc):
    recs = [oracle_record(orc, m) for m in range(2, 8)] + [golden_record(9), golden_record(10)]
    with rd.Server(hbm_budget_bytes=8 << 30) as sv:
        for r in recs:
            sv.import_relation(r)
        assert sv.export_relation(9) == recs[-2]
        assert sv.export_relation(8) is None  # nothing recorded, nothing searched
        import numpy as np

        rng = np.random.default_rng(7)
        ms = rng.choice([r["m"] for r in recs], size=2000)
        ns = rng.integers(3, 5000, size=2000)
        t = sv.submit(ms, ns)
        g, st, _ = sv.wait(t, timeout_s=60)
        by_m = {r["m"]: r for r in recs}
        assert (st == rd.RD_OK).all()
        for m, n, got in zip(ms, ns, g):
            assert got == closed_form(by_m[int(m)], int(n)), (m, n)
        s = sv.stats()
        assert s["jobs_admitted"] == 0 and s["bytes_peak"] == 0  # every answer came from a record


def test_server_export_after_a_search(rd, orc):
    with rd.Server(hbm_budget_bytes=8 << 30) as sv:
        g, st, _ = sv.wait(sv.submit([5, 6], [40, 41]), timeout_s=120)
        assert (st == rd.RD_OK).all()
        for m in (5, 6):
            assert sv.export_relation(m) == oracle_record(orc, m), m
        with pytest.raises(rd.RdError) as e:
            sv.import_relation(dict(oracle_record(orc, 5), q=13))  # gamma[k + p] != gamma[k] + q
        assert e.value.status == rd.RD_ERR_ARG


def test_server_import_while_its_search_runs(rd, orc):
    """A record imported for an m whose search is already running: queries routed after the import are
    answered from it, the running search still completes, and every answer (before, during and after)
    equals Prop. 7 from the oracle's first repeat."""
    import numpy as np

    rec = golden_record(9)
    with rd.Server(hbm_budget_bytes=32 << 30) as sv:
        first = sv.submit([9] * 4, [30, 31, 500, 1001])  # starts the m = 9 search
        sv.import_relation(rec)
        second = sv.submit([9] * 4, [3, 27, 28, 12345])
        g, st, _ = sv.wait(np.concatenate([first, second]), timeout_s=120)
        assert (st == rd.RD_OK).all()
        ns = [30, 31, 500, 1001, 3, 27, 28, 12345]
        assert [int(x) for x in g] == [closed_form(rec, n) for n in ns]
        assert sv.export_relation(9) == rec
