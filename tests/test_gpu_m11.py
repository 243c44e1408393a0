"""m = 11 (N = 191,476; one power is 73 GB): the period search on one GPU in low memory.

Three ring slots (220 GB) with A(G) built in the first (it is read only for the first power), the
row split's intermediate in 8192-column chunks, and the repeat verified by re-deriving the earlier
power when it has left the ring.  The paper has no m = 11 row in Table 2; what it fixes: Cor. 12
(gamma = 2(m + 1) n / 5 = 24 n / 5 for n = 0 mod 5, n >= 10), Remark 13 (the same at n = 5),
Theorem 11's lower bound ceil(24 n / 5) for n >= 10, and the path DP for small n.  The oracle cannot run
the m = 11 search, but it computes single rows of A^k from the arc lists (about a minute for the lists):
sampled rows of the last power are compared with them.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

INF64 = 0x3FFFFFFFFFFFFFFF
I16_INF = 0x3FFF


@pytest.fixture(scope="module")
def rd():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    return rd


def check_m11_gamma(orc, gamma_of, j):
    for n in range(3, 7):
        assert gamma_of(n) == orc.row_dp(11, n), n
    assert gamma_of(5) == 24  # Remark 13
    for n in range(10, j + 1):
        assert gamma_of(n) >= math.ceil(24 * n / 5), n  # Theorem 11
        if n % 5 == 0:
            assert 5 * gamma_of(n) == 24 * n, n  # Cor. 12


def test_m11_search_low_memory(rd, orc):
    import torch

    torch.cuda.empty_cache()
    m, kmax = 11, 48
    n = rd.state_count(m)
    ld = rd.padded_dim(n)
    work = rd.power_workspace(n, ld, kmax, 3)
    off0 = rd.power_slot(n, ld, kmax, work.numel(), 0)
    A = work[off0:off0 + n * ld * 2].view(torch.int16).view(n, ld)
    rd.build_transfer(m, A)
    plan = rd.split_plan(m, chunk_cols=8192)
    r = rd.power_until_periodic_split(A, plan, kmax, work)
    assert r["found"], r["status"]
    # sampled rows of the last power P_j (its slot is left alone by the re-derivation) against the oracle's
    # rows of A^j and A^k: equal up to one constant each, so A^(k+p) = q (x) A^k holds on those rows too
    j, k = r["j"], r["k"]
    off = rd.power_slot(n, ld, kmax, work.numel(), j)
    rows = np.array([0, 1, n // 2, n - 1])
    pj = work[off:off + n * ld * 2].view(torch.int16).view(n, ld)[rows.tolist(), :n].cpu().numpy().astype(np.int64)
    del A, work, plan
    torch.cuda.empty_cache()
    ora = orc.power_rows(m, rows, j)  # rows of A^1..A^j from the arc lists (raw int64)
    diffs = []
    for kk in (j, k):
        want = ora[kk - 1]
        fin = want != INF64
        assert np.array_equal(pj == I16_INF, ~fin), kk
        d = want[fin] - pj[fin]
        assert np.all(d == d[0]), kk
        diffs.append(int(d[0]))
    assert diffs[0] - diffs[1] == r["q"]
    g = r["gamma"]
    check_m11_gamma(orc, lambda nn: int(g[nn]), r["j"])
    # the relation continues Cor. 12: over one period gamma grows by 24 n / 5 per 5 columns
    assert r["q"] * 5 == 24 * r["p"], (r["k"], r["p"], r["q"])


def test_m11_gamma_R(rd, orc):
    import torch

    torch.cuda.empty_cache()
    check_m11_gamma(orc, lambda nn: rd.gamma_R(11, nn), 60)
    assert rd.gamma_R(11, 1000) == 4800
