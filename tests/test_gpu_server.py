"""The query server: answers equal those computed alone (and the oracle), admission by HBM footprint,
and its error paths.  GPU only."""
import math
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    return rd


def expected(orc, cache, m, n):
    if m not in cache:
        r = orc.power_until_periodic(m, kmax=48)
        cache[m] = r
    r = cache[m]
    return orc.gamma_from_period(r["gamma"], r["k"], r["p"], r["q"], n)


def test_server_mix_equals_alone(rd, orc):
    rng = np.random.default_rng(5)
    ms = rng.integers(1, 10, 600).astype(np.int32)
    ns = rng.integers(3, 201, 600).astype(np.int64)
    with rd.Server(hbm_budget_bytes=64 << 30, kmax=128) as sv:
        tickets = []
        # bursts: later queries arrive while earlier searches are on the GPU
        for lo in range(0, 600, 100):
            tickets.append(sv.submit(ms[lo:lo + 100], ns[lo:lo + 100]))
            time.sleep(0.01)
        g, st, lat = sv.wait(np.concatenate(tickets), timeout_s=600)
        stats = sv.stats()
    assert np.all(st == rd.RD_OK)
    assert np.all(lat >= 0)
    cache = {}
    for m, n, v in zip(ms, ns, g):
        assert v == rd.gamma_R(int(m), int(n)), (m, n)  # the same query answered alone
        if m <= 6:
            assert v == expected(orc, cache, int(m), int(n)), (m, n)
        if m == 1:
            assert v == math.ceil(2 * n / 3)
    assert stats["jobs_completed"] == len(set(ms.tolist()))
    assert stats["answered"] == 600 and stats["bytes_in_use"] == 0


def test_server_concurrent_submitters(rd):
    out = {}

    def client(idx, sv):
        rng = np.random.default_rng(100 + idx)
        ms = rng.integers(2, 9, 50).astype(np.int32)
        ns = rng.integers(3, 120, 50).astype(np.int64)
        g, st, _ = sv.wait(sv.submit(ms, ns), timeout_s=600)
        out[idx] = (ms, ns, g, st)

    with rd.Server(hbm_budget_bytes=16 << 30, kmax=128) as sv:
        th = [threading.Thread(target=client, args=(i, sv)) for i in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    for ms, ns, g, st in out.values():
        assert np.all(st == rd.RD_OK)
        for m, n, v in zip(ms, ns, g):
            assert v == rd.gamma_R(int(m), int(n))


def test_server_admission_by_footprint(rd):
    # m = 9 alone needs ~8.7 GB (A, 8 powers, plan); with a 9.5 GB budget m = 8 (~1 GB) must wait for it
    budget = int(9.5 * (1 << 30))
    with rd.Server(hbm_budget_bytes=budget, kmax=64) as sv:
        t = sv.submit([9, 8, 7, 9, 8], [40, 41, 42, 5, 6])
        g, st, _ = sv.wait(t, timeout_s=600)
        stats = sv.stats()
    assert np.all(st == rd.RD_OK)
    assert list(g) == [rd.gamma_R(9, 40), rd.gamma_R(8, 41), rd.gamma_R(7, 42), rd.gamma_R(9, 5), rd.gamma_R(8, 6)]
    assert stats["bytes_peak"] <= budget and stats["jobs_completed"] == 3


def test_server_errors(rd):
    with rd.Server(hbm_budget_bytes=256 << 20, kmax=64) as sv:
        with pytest.raises(rd.RdError) as e:
            sv.submit([0], [5])
        assert e.value.status == rd.RD_ERR_ARG
        with pytest.raises(rd.RdError) as e:
            sv.submit([3], [2])
        assert e.value.status == rd.RD_ERR_ARG
        # m = 9 cannot fit a 256 MiB budget: its queries fail with RD_ERR_NOMEM, others still work
        g, st, _ = sv.wait(sv.submit([9, 3], [10, 10]), timeout_s=120)
        assert st[0] == rd.RD_ERR_NOMEM and st[1] == rd.RD_OK and g[1] == rd.gamma_R(3, 10)
        # a wait that runs out returns RD_ERR_TIMEOUT and keeps the ticket
        t = sv.submit([7], [150])
        try:
            sv.wait(t, timeout_s=0.0)
        except rd.RdError as err:
            assert err.status == rd.RD_ERR_TIMEOUT
        g, st, _ = sv.wait(t, timeout_s=120)
        assert st[0] == rd.RD_OK and g[0] == rd.gamma_R(7, 150)
