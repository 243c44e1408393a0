"""The autotuners (rd_tune_gemm, rd_tune_split, rd_sparse_tune) and the launchers that read their
table, on a GB300: a tuned launch shape changes time only, so every product and period search run
with a table entry stays bit-exact against the CPU oracle."""
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


@pytest.fixture(autouse=True)
def empty_table(rd):
    rd.tune_set([])
    yield
    rd.tune_set([])


def to_i16(a64):
    return np.where(a64 == INF64, I16_INF, a64).astype(np.int16)


def upload(torch, host):
    rows, cols = host.shape
    t = torch.full((rows, (cols + 7) // 8 * 8), -3, dtype=torch.int16)  # junk padding the kernels must not read
    t[:, :cols] = torch.from_numpy(np.ascontiguousarray(host))
    return t.cuda()


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("S", [1, 2, 4, 8])
def test_gemm_reads_its_split_factor_from_the_table(rd, orc, S, tile):
    """Every split factor with both output tiles (128 x 256 and 128 x 128), on a ragged product."""
    import torch
    from paper_2409_17658_gb300 import inputs

    M, N, K = 257, 300, 1500
    a = inputs.matrix(M, K, seed=41, dist="wide")
    b = inputs.matrix(K, N, seed=42, dist="wide")
    A, B = upload(torch, a), upload(torch, b)
    C = torch.full((M, B.shape[1]), 777, dtype=torch.int16, device="cuda")
    rd.tune_set([dict(mode="gemm_splitk", key=rd.tune_bucket(max(M, N)), aux=rd.tune_bucket(K), p=[S, tile, 0, 0])])
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.minplus_gemm(A, B, C, M, N, K, min_out=mn)
    want = orc.minplus_i16(a, b)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :N].astype(np.int32), want) and np.all(got[:, N:] == 777)
    assert mn.item() == want.min()


def test_gemm_table_factor_that_does_not_suit_falls_back(rd, orc):
    """S = 8 on K = 200 would leave empty K slices: the launcher ignores the entry."""
    import torch
    from paper_2409_17658_gb300 import inputs

    M, N, K = 130, 140, 200
    a = inputs.matrix(M, K, seed=43, dist="u32")
    b = inputs.matrix(K, N, seed=44, dist="u32")
    A, B = upload(torch, a), upload(torch, b)
    C = torch.empty((M, B.shape[1]), dtype=torch.int16, device="cuda")
    rd.tune_set([dict(mode="gemm_splitk", key=rd.tune_bucket(N), aux=rd.tune_bucket(K), p=[8, 0, 0, 0])])
    rd.minplus_gemm(A, B, C, M, N, K)
    assert np.array_equal(C.cpu().numpy()[:, :N].astype(np.int32), orc.minplus_i16(a, b))


def test_tune_gemm_records_the_fastest_factor(rd, orc):
    import torch
    from paper_2409_17658_gb300 import inputs

    n = 1024
    A = inputs.matrix_torch(n, n, seed=1, dist="u32", device="cuda")
    B = inputs.matrix_torch(n, n, seed=2, dist="u32", device="cuda")
    C = torch.empty((n, n), dtype=torch.int16, device="cuda")
    e = rd.tune_gemm(A, B, C, reps=3)
    assert e["mode"] == "gemm_splitk" and e["key"] == 10 and e["aux"] == 10 and e["p"][0] in (1, 2, 4, 8)
    assert e["p"][1] in (0, 1)
    assert e["ms"] > 0 and rd.tune_table() == [e]
    rd.minplus_gemm(A, B, C)  # with the recorded factor
    a, b = A.cpu().numpy(), B.cpu().numpy()
    assert np.array_equal(C.cpu().numpy().astype(np.int32), orc.minplus_i16(a, b))


@pytest.mark.parametrize("n", [1024, 2048])
def test_narrow_tile_at_sweep_sizes(rd, orc, n):
    """The 128 x 128 tile (no split and split by 4) on the sweep's small sizes: all entries against the oracle."""
    import torch
    from paper_2409_17658_gb300 import inputs

    A = inputs.matrix_torch(n, n, seed=5, dist="wide", device="cuda")
    B = inputs.matrix_torch(n, n, seed=6, dist="wide", device="cuda")
    a, b = A.cpu().numpy(), B.cpu().numpy()
    want = orc.minplus_i16(a, b) if n <= 1024 else None
    rng = np.random.default_rng(n)
    ri, cj = rng.integers(0, n, 256), rng.integers(0, n, 256)
    for S in (1, 4):
        rd.tune_set([dict(mode="gemm_splitk", key=rd.tune_bucket(n), aux=rd.tune_bucket(n), p=[S, 1, 0, 0])])
        C = torch.empty((n, n), dtype=torch.int16, device="cuda")
        mn = torch.zeros(1, dtype=torch.int32, device="cuda")
        rd.minplus_gemm(A, B, C, min_out=mn)
        got = C.cpu().numpy().astype(np.int32)
        if want is not None:
            assert np.array_equal(got, want) and mn.item() == want.min(), S
        else:
            assert np.array_equal(got[ri, cj], orc.minplus_i16_entries(a, b, ri, cj)), S


def test_tune_gemm_argument_checks(rd):
    import torch

    A = torch.zeros((8, 8), dtype=torch.int16, device="cuda")
    for args in [(A, A, A, 1, 8, 8), (A, A, A, 8, 8, 0), (A, A, A, 8, 8, 16)]:
        with pytest.raises(rd.RdError):
            rd.tune_gemm(*args)
    assert rd.tune_table() == []


def test_tune_split_m7_then_plans_and_searches_use_it(rd, orc):
    import torch
    from paper_2409_17658_gb300 import inputs

    m = 7
    n = rd.state_count(m)
    b = inputs.matrix(n, n, seed=97, dist="wide")
    B = upload(torch, b)
    C = torch.empty_like(B)
    plan = rd.split_plan(m)
    before = plan["info"].as_dict()
    e = rd.tune_split(plan, B, C, reps=2)
    info = plan["info"]
    assert e["mode"] == "split" and (e["key"], e["aux"]) == (m, info.j)
    assert e["p"] == [info.w1, info.k1, info.w2, info.k2] and e["ms"] > 0
    # the tuned plan computes the same product
    rd.split_minplus(plan, B, C)
    rng = np.random.default_rng(7)
    ri = np.concatenate([[0, n - 1], rng.integers(0, n, 300)])
    cj = np.concatenate([[n - 1, 0], rng.integers(0, n, 300)])
    want = orc.minplus_i16_entries(to_i16(orc.transfer_rows(m, np.arange(n))), b, ri, cj)
    assert np.array_equal(C.cpu().numpy()[ri, cj].astype(np.int32), want)
    # a new plan for (m, j) takes the tuned shape; every other field is the built-in plan's
    plan2 = rd.split_plan(m)
    got = plan2["info"].as_dict()
    assert [got["w1"], got["k1"], got["w2"], got["k2"]] == e["p"]
    for f in before:
        if f not in ("w1", "k1", "w2", "k2"):
            assert got[f] == before[f], f
    # and the period search through it is Table 2's (21, 5, 16) with the oracle's gamma
    A, _ = rd.transfer_matrix(m)
    work = rd.power_workspace(n, A.stride(0), 32, 8)
    r = rd.power_until_periodic_split(A, plan2, 32, work)
    o = orc.power_until_periodic(m, kmax=32)
    assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"]) == (21, 5, 16)
    assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1])


@pytest.mark.parametrize("shape", [(32, 1), (64, 64), (128, 2), (32, 32), (256, 1), (256, 16)])
def test_split_shapes_from_the_table_are_bit_exact(rd, orc, shape):
    """Every width and slabs-per-CTA the tuner may pick, installed through the table, at m = 6."""
    import torch
    from paper_2409_17658_gb300 import inputs

    m = 6
    j = rd.split_default_j(m)
    w, k = shape
    rd.tune_set([dict(mode="split", key=m, aux=j, p=[w, k, w, k])])
    plan = rd.split_plan(m)
    assert (plan["info"].w1, plan["info"].k1, plan["info"].w2, plan["info"].k2) == (w, k, w, k)
    n = rd.state_count(m)
    b = inputs.matrix(n, n, seed=66, dist="wide")
    B = upload(torch, b)
    C = torch.empty_like(B)
    rd.split_minplus(plan, B, C)
    a = orc.transfer(m)
    assert np.array_equal(C.cpu().numpy()[:, :n].astype(np.int32), orc.minplus_i16(to_i16(a), b))


def test_sparse_tune_records_its_r(rd):
    m = 7
    A, n = rd.transfer_matrix(m)
    work = rd.power_workspace(n, A.stride(0), 8, 8)
    best, ms = rd.sparse_tune(A, n, work)
    e = rd.tune_lookup(rd.RD_TUNE_SPARSE_R, rd.tune_bucket(n), 0)
    assert e is not None and e["p"][0] == best and best in ms


def test_server_with_tuned_split_shapes(rd, orc):
    """A server whose m = 8 and m = 9 jobs build their row-split plans from tuning-table shapes (narrow slabs,
    one slab per CTA) answers as the oracle's relation says (m = 8) and as Table 2 implies (m = 9)."""
    rd.tune_set([dict(mode="split", key=8, aux=4, p=[32, 1, 32, 1]), dict(mode="split", key=9, aux=4, p=[64, 2, 32, 4])])
    ns = np.arange(3, 61, dtype=np.int64)
    ms = np.array([8] * len(ns) + [9] * len(ns), dtype=np.int32)
    with rd.Server(hbm_budget_bytes=64 << 30, kmax=64) as sv:
        g, st, _ = sv.wait(sv.submit(ms, np.concatenate([ns, ns])), timeout_s=600)
    assert np.all(st == rd.RD_OK)
    o8 = orc.power_until_periodic(8, kmax=48)
    want8 = [orc.gamma_from_period(o8["gamma"], o8["k"], o8["p"], o8["q"], int(n)) for n in ns]
    assert list(g[:len(ns)]) == want8
    # m = 9: Table 2's relation (22, 5, 20) and Remark 13 (gamma = 2(m + 1)n/5 for n = 0 mod 5)
    g9 = dict(zip(ns.tolist(), g[len(ns):].tolist()))
    for n in range(30, 61):
        assert g9[n] == g9[n - 5] + 20, n
    for n in range(5, 61, 5):
        assert 5 * g9[n] == 2 * 10 * n, n
