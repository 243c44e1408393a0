"""Parity of the row-split power step (rd_split_*) with the CPU oracle, on a GB300.

The row-split step forms R = A(G) (x) B from the row rules of Sec. 4.A in two
passes, without A(G).  Every comparison is bit-exact against the oracle's
products with A(G) built from the definition, or against the oracle's own
period search; seeded operands come from paper_2409_17658_gb300.inputs.
"""
import os

import numpy as np
import pytest

from conftest import oracle_first_repeat, oracle_m9, read_golden

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

    checked = os.environ.get("RD_CHECKED_LIB")  # set by test_gpu_split_checked.py: run under the checked build
    prev = rd.use_library(checked) if checked else None
    yield rd
    if checked:
        rd.use_library_handle(prev)


@pytest.fixture(autouse=True)
def no_index_violations(rd):
    """Under the checked build, no test may leave an index-check bit set (rd_split_check_flags)."""
    rd.split_check_flags(reset=True)
    yield
    import torch

    torch.cuda.synchronize()
    assert rd.split_check_flags(reset=True) in (None, 0)


@pytest.fixture(scope="module")
def torch_mod():
    import torch

    return torch


def to_i16(a64):
    return np.where(a64 == INF64, I16_INF, a64).astype(np.int16)


def upload(torch, host, junk):
    rows, cols = host.shape
    ld = (cols + 7) // 8 * 8
    t = torch.full((rows, ld), junk, dtype=torch.int16)
    t[:, :cols] = torch.from_numpy(np.ascontiguousarray(host))
    return t.cuda()


def type_counts(orc, m, j):
    """(distinct row-type prefixes of rows 1..j, suffixes of rows j+1..m) over the correct words, by brute force."""
    codes = orc.words(m)[0]

    def letter(c, i):
        return (int(c) >> (2 * (m - i))) & 3

    def rtype(c, i):
        x = letter(c, i)
        if x != 2:
            return "abXd"[x]
        vert = (i > 1 and letter(c, i - 1) == 0) or (i < m and letter(c, i + 1) == 0)
        return "+" if vert else "-"

    types = ["".join(rtype(c, i) for i in range(1, m + 1)) for c in codes]
    return len({t[:j] for t in types}), len({t[j:] for t in types})


SMALL = [(m, j) for m in range(2, 7) for j in range(1, m)]


@pytest.mark.parametrize("m,j", SMALL)
def test_split_minplus_matches_oracle(rd, torch_mod, orc, m, j):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    n = rd.state_count(m)
    b = inputs.matrix(n, n, seed=70 + m, dist="wide")
    B = upload(torch, b, junk=-5)  # padding columns hold junk the kernels must not use
    plan = rd.split_plan(m, j)
    info = plan["info"]
    assert (info.m, info.j, info.N) == (m, j, n)
    assert (info.n_rho, info.n_sigma) == type_counts(orc, m, j)
    assert (info.n_pi, info.n_phi) == (rd.state_count(j), rd.state_count(m - j))
    assert 0 < info.x_rows <= info.n_pi * info.n_sigma
    assert 0 < info.slots1 <= info.n_pi and 0 < info.slots2 <= info.n_sigma
    C = torch.full((n, B.stride(0)), 777, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.split_minplus(plan, B, C, min_out=mn)
    want = orc.minplus_i16(to_i16(orc.transfer(m)), b)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :n].astype(np.int32), want)
    assert np.all(got[:, n:] == 777)
    assert mn.item() == want.min()


def test_split_minplus_all_infinite_and_slab_widths(rd, torch_mod, orc):
    """B = all RD_INF gives RD_INF everywhere (min_out RD_INF); every slab width gives the same product."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    m = 5
    n = rd.state_count(m)
    plan = rd.split_plan(m)
    B = torch.full((n, rd.padded_dim(n)), I16_INF, dtype=torch.int16, device="cuda")
    C = torch.zeros_like(B)
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.split_minplus(plan, B, C, min_out=mn)
    assert bool((C[:, :n] == I16_INF).all()) and mn.item() == I16_INF
    b = inputs.matrix(n, n, seed=80, dist="u32")
    B = upload(torch, b, junk=I16_INF)
    want = orc.minplus_i16(to_i16(orc.transfer(m)), b)
    for w1 in (32, 64, 128, 256):
        for w2 in (32, 64, 128, 256):
            plan["info"].w1, plan["info"].w2 = w1, w2
            C.fill_(0)
            rd.split_minplus(plan, B, C)
            assert np.array_equal(C[:, :n].cpu().numpy().astype(np.int32), want), (w1, w2)


@pytest.mark.parametrize("m", [7, 8])
def test_split_minplus_sampled(rd, torch_mod, orc, m):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    n = rd.state_count(m)
    b = inputs.matrix(n, n, seed=90 + m, dist="wide")
    B = upload(torch, b, junk=-5)
    C = torch.empty_like(B)
    for j in range(max(1, m - 8), min(m - 1, 8) + 1):
        plan = rd.split_plan(m, j)
        rd.split_minplus(plan, B, C)
        rng = np.random.default_rng(m * 10 + j)
        ri = np.concatenate([[0, n - 1, n - 1], rng.integers(0, n, 400)])
        cj = np.concatenate([[0, n - 1, 0], rng.integers(0, n, 400)])
        want = orc.minplus_i16_entries(to_i16(orc.transfer_rows(m, np.arange(n))), b, ri, cj)
        got = C.cpu().numpy()[ri, cj].astype(np.int32)
        assert np.array_equal(got, want), j


def test_split_minplus_m10_full_size_sampled(rd, torch_mod, orc):
    """m = 10 (N = 64769) in the launch configuration of the period search; sampled entries from the
    oracle's rows of A(G) and the generator's own entries of B."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    m, seed = 10, 123
    n = rd.state_count(m)
    ld = rd.padded_dim(n)
    B = inputs.matrix_torch(n, n, seed, dist="wide", ld=ld, device="cuda")
    plan = rd.split_plan(m)
    C = torch.empty_like(B)
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.split_minplus(plan, B, C, min_out=mn)
    rng = np.random.default_rng(1010)
    rows = np.concatenate([[0, n - 1], rng.integers(0, n, 6)])
    cols = np.concatenate([[0, n - 1, 7, 8, n - 2], rng.integers(0, n, 59)])
    arows = orc.transfer_rows(m, rows)
    got = C[rows.tolist()][:, cols.tolist()].cpu().numpy().astype(np.int64)
    for r in range(len(rows)):
        ts = np.nonzero(arows[r] != INF64)[0]
        for c, col in enumerate(cols):
            bv = inputs.entries(ts, np.full(len(ts), col), n, seed, "wide").astype(np.int64)
            v = np.where(bv == I16_INF, I16_INF, arows[r][ts] + bv)
            assert got[r, c] == min(I16_INF, int(v.min())), (rows[r], col)
    assert 0 <= mn.item() <= int(got.min())
    del B, C, plan
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- period search with the row-split step

@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7])
def test_power_split_matches_oracle(rd, torch_mod, orc, m):
    A, n = rd.transfer_matrix(m)
    plan = rd.split_plan(m)
    work = rd.power_workspace(n, A.stride(0), 48, 8)
    r = rd.power_until_periodic_split(A, plan, 48, work)
    o = orc.power_until_periodic(m, kmax=48)
    assert r["found"] and o["found"]
    assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"])
    assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1])
    assert np.all(r["gamma"][r["j"] + 1:] == rd.RD_GAMMA_UNSET)
    if m <= 5:
        # the resident powers are A^k - o_k exactly
        a = orc.transfer(m)
        powers = {1: a}
        for k in range(2, r["j"] + 1):
            powers[k] = orc.power_step(powers[k - 1], a)
        ld = A.stride(0)
        raw = work.cpu().numpy()
        for k in range(r["j"] - 7, r["j"] + 1):
            off = rd.power_slot(n, ld, 48, work.numel(), k)
            pk = raw[off:off + n * ld * 2].view(np.int16).reshape(n, ld)[:, :n]
            want = powers[k]
            fin = want[want != INF64]
            assert np.array_equal(pk, to_i16(np.where(want == INF64, INF64, want - fin.min()))), k


@pytest.mark.parametrize("m,kmax", [(5, 17), (5, 20), (7, 9), (7, 25)])
def test_power_split_not_found_within_kmax(rd, torch_mod, orc, m, kmax):
    """The row-split search stopped by kmax one power short of its repeat (and far short of it): RD_NOT_FOUND,
    with gamma[1..kmax] equal to the oracle's, and the same workspace then finds the relation."""
    torch = torch_mod
    A, n = rd.transfer_matrix(m)
    plan = rd.split_plan(m)
    work = rd.power_workspace(n, A.stride(0), 48, 8)
    r = rd.power_until_periodic_split(A, plan, kmax, work)
    assert r["status"] == rd.RD_NOT_FOUND and not r["found"]
    want = orc.power_until_periodic(m, kmax=48)["gamma"]
    assert [int(x) for x in r["gamma"][1:kmax + 1]] == [int(x) for x in want[1:kmax + 1]]
    r2 = rd.power_until_periodic_split(A, plan, 48, work)
    assert r2["found"] and r2["j"] > kmax
    del work, plan, A
    torch.cuda.empty_cache()


def test_power_split_m8_matches_oracle(rd, torch_mod, orc):
    A, n = rd.transfer_matrix(8)
    plan = rd.split_plan(8)
    work = rd.power_workspace(n, A.stride(0), 30, 8)
    r = rd.power_until_periodic_split(A, plan, 30, work)
    o = orc.power_until_periodic(8, kmax=30)
    assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"]) == (21, 5, 18)
    assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1])


def test_power_split_m9(rd, torch_mod, orc):
    """m = 9 (N = 21909): the oracle's first repeat and gamma[1..j], Table 2's triple, the path DP for n <= 7,
    sampled rows of the resident powers against the oracle, and the same gamma sequence and final power as
    the sparse step."""
    torch = torch_mod
    m, kmax, slots = 9, 40, 8
    A, n = rd.transfer_matrix(m)
    ld = A.stride(0)
    plan = rd.split_plan(m)
    work = rd.power_workspace(n, ld, kmax, slots)
    r = rd.power_until_periodic_split(A, plan, kmax, work)
    table = {int(x[0]): tuple(map(int, x[1:])) for x in read_golden("paper_table2_periods.txt")}
    assert r["found"] and (r["k"], r["p"], r["q"]) == table[9]
    o = oracle_m9()  # the oracle's row-streamed first-repeat search
    assert (r["k"], r["p"], r["q"], r["j"]) == (o["k"], o["p"], o["q"], o["j"])
    assert [int(x) for x in r["gamma"][1:r["j"] + 1]] == o["gamma"][1:o["j"] + 1]
    for nn in range(3, 8):
        assert r["gamma"][nn] == orc.row_dp(m, nn)
    rng = np.random.default_rng(909)
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 10)]))
    ora = orc.power_rows(m, rows, r["j"])
    for k in range(r["j"] - slots + 1, r["j"] + 1):
        off = rd.power_slot(n, ld, kmax, work.numel(), k)
        pk = work[off:off + n * ld * 2].view(torch.int16).view(n, ld)[rows.tolist(), :n].cpu().numpy()
        want = ora[k - 1]
        fin = want != INF64
        assert np.array_equal(pk == I16_INF, ~fin)
        d = want[fin] - pk[fin].astype(np.int64)
        assert np.all(d == d[0]) and pk[fin].min() >= 0, k
    sp = rd.sparse_plan(A, n, n, 2)
    work2 = rd.power_workspace(n, ld, kmax, slots)
    s = rd.power_until_periodic_sparse(A, n, sp, kmax, work2)
    assert np.array_equal(r["gamma"], s["gamma"])
    off = rd.power_slot(n, ld, kmax, work.numel(), r["j"])
    off2 = rd.power_slot(n, ld, kmax, work2.numel(), s["j"])
    assert torch.equal(work[off:off + n * ld * 2].view(torch.int16).view(n, ld)[:, :n],
                       work2[off2:off2 + n * ld * 2].view(torch.int16).view(n, ld)[:, :n])


def test_power_split_m10(rd, torch_mod, orc):
    """m = 10 (N = 64769): the oracle's first repeat and gamma[1..j] (its row-streamed search, stored), Cor. 12
    (gamma = 22n/5 for n = 0 mod 5, n >= 10), Remark 13 (n = 5),
    Theorem 11's lower bound, the path DP for n <= 7, and sampled rows of the resident powers."""
    torch = torch_mod
    m, kmax = 10, 48
    A, n = rd.transfer_matrix(m)
    ld = A.stride(0)
    plan = rd.split_plan(m)
    work = rd.power_workspace(n, ld, kmax, 8)
    r = rd.power_until_periodic_split(A, plan, kmax, work)
    assert r["found"]
    g = r["gamma"]
    o = oracle_first_repeat(10)  # the oracle's row-streamed first-repeat search
    assert (r["k"], r["p"], r["q"], r["j"]) == (o["k"], o["p"], o["q"], o["j"])
    assert [int(x) for x in g[1:r["j"] + 1]] == o["gamma"][1:o["j"] + 1]

    def gamma(nn):
        if nn <= r["j"]:
            return int(g[nn])
        k, p, q = r["k"], r["p"], r["q"]
        return int(g[k + (nn - k) % p]) + q * ((nn - k) // p)

    for nn in range(3, 8):
        assert gamma(nn) == orc.row_dp(m, nn), nn
    assert gamma(5) == 22
    for nn in range(10, 401):
        assert 5 * gamma(nn) >= 22 * nn, nn
        if nn % 5 == 0:
            assert 5 * gamma(nn) == 22 * nn, nn
    rng = np.random.default_rng(1011)
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 2)]))
    ora = orc.power_rows(m, rows, r["j"])
    for k in range(r["j"] - 2, r["j"] + 1):
        off = rd.power_slot(n, ld, kmax, work.numel(), k)
        pk = work[off:off + n * ld * 2].view(torch.int16).view(n, ld)[rows.tolist(), :n].cpu().numpy()
        want = ora[k - 1]
        fin = want != INF64
        assert np.array_equal(pk == I16_INF, ~fin)
        d = want[fin] - pk[fin].astype(np.int64)
        assert np.all(d == d[0]), k
    del work, plan, A
    torch.cuda.empty_cache()


@pytest.mark.parametrize("graph_steps", [0, 8])
def test_power_multi_mixes_split_and_sparse_runs(rd, torch_mod, orc, graph_steps):
    """rd_power_until_periodic_multi with row-split runs (even m) beside sparse runs (odd m), with and
    without the CUDA graph: each run's relation and gamma sequence equal the oracle's (m <= 7) and
    Table 2 (m = 8, 9)."""
    kmax = 48
    runs = []
    for m in range(1, 10):
        A, n = rd.transfer_matrix(m)
        plan = rd.split_plan(m, x_ld=A.stride(0)) if m % 2 == 0 else rd.sparse_plan(A, n, n, 2)
        runs.append((A, n, plan, rd.power_workspace(n, A.stride(0), kmax, 8)))
    res = rd.power_until_periodic_multi(runs, 2, kmax, graph_steps=graph_steps)
    table = {int(x[0]): tuple(map(int, x[1:])) for x in read_golden("paper_table2_periods.txt")}
    for m, r in zip(range(1, 10), res):
        assert r["found"], m
        if m <= 7:
            o = orc.power_until_periodic(m, kmax=kmax)
            assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"]), m
            assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1]), m
        if m in table:  # the first repeat implies the printed relation (at m = 4 its period 1 divides 5)
            n0, alpha, beta = table[m]
            assert n0 >= r["k"] and alpha % r["p"] == 0 and beta == r["q"] * (alpha // r["p"]), m
    for nn in range(3, 8):
        assert res[8]["gamma"][nn] == orc.row_dp(9, nn)
    o9 = oracle_m9()
    assert (res[8]["k"], res[8]["p"], res[8]["q"]) == (o9["k"], o9["p"], o9["q"])
    assert [int(x) for x in res[8]["gamma"][1:res[8]["j"] + 1]] == o9["gamma"][1:o9["j"] + 1]


@pytest.mark.parametrize("m", [7, 9])
def test_power_split_short_ring_rederives(rd, torch_mod, orc, m):
    """A ring of 3 slots is shorter than the period (5): when P_(k+p)'s hash matches P_k, P_k has left the ring,
    so the search stops, re-derives P_k from A(G) in the two spare slots and compares it with P_(k+p) entry by
    entry.  The relation and gamma equal the oracle's (m = 9: its row-streamed search)."""
    kmax = 40
    A, n = rd.transfer_matrix(m)
    plan = rd.split_plan(m, x_ld=A.stride(0))
    work = rd.power_workspace(n, A.stride(0), kmax, 3)
    r = rd.power_until_periodic_split(A, plan, kmax, work)
    if m == 7:
        o = orc.power_until_periodic(m, kmax=kmax)
        want_gamma = [int(x) for x in o["gamma"][1:o["j"] + 1]]
    else:
        o = oracle_m9()
        want_gamma = o["gamma"][1:o["j"] + 1]
    assert r["found"] and (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"])
    assert [int(x) for x in r["gamma"][1:r["j"] + 1]] == want_gamma


@pytest.mark.parametrize("j", [1, 2, 5, 6])
def test_power_split_every_split_point_m7(rd, torch_mod, orc, j):
    """The period search through unbalanced splits (fibers of up to 1085 slots, metadata read from global
    memory where it does not fit beside the rows) gives the oracle's relation and gamma sequence."""
    m = 7
    A, n = rd.transfer_matrix(m)
    plan = rd.split_plan(m, j, x_ld=A.stride(0))
    r = rd.power_until_periodic_split(A, plan, 40, rd.power_workspace(n, A.stride(0), 40, 8))
    o = orc.power_until_periodic(m, kmax=40)
    assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"])
    assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1])


@pytest.mark.parametrize("chunk", [128, 384, 1024])
def test_split_column_chunks(rd, torch_mod, orc, chunk):
    """chunk_cols > 0: both passes run chunk by chunk with X holding one chunk (ragged last chunk
    included); the product and the period search equal the oracle's."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    m = 6
    n = rd.state_count(m)
    b = inputs.matrix(n, n, seed=111, dist="wide")
    B = upload(torch, b, junk=-5)
    plan = rd.split_plan(m, chunk_cols=chunk)
    assert plan["X"].shape[1] == chunk
    C = torch.full((n, B.stride(0)), 777, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.split_minplus(plan, B, C, min_out=mn)
    want = orc.minplus_i16(to_i16(orc.transfer(m)), b)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :n].astype(np.int32), want)
    assert np.all(got[:, n:] == 777) and mn.item() == want.min()
    A, _ = rd.transfer_matrix(m)
    r = rd.power_until_periodic_split(A, plan, 40, rd.power_workspace(n, A.stride(0), 40, 8))
    o = orc.power_until_periodic(m, kmax=40)
    assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"])
    assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1])
