"""Parity of the CUDA path (through the C ABI) with the CPU oracle, on a GB300.

Integer work throughout, so every comparison is bit-exact.  Inputs are the
transfer matrices of the paper (from the definition) and seeded synthetic
operands from paper_2409_17658_gb300.inputs.
"""
import math

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

    return rd


@pytest.fixture(scope="module")
def torch_mod():
    import torch

    return torch


def to_i16(a64):
    return np.where(a64 == INF64, I16_INF, a64).astype(np.int16)


def upload(torch, host, ld=None, junk=None):
    """Copy a host int16 matrix into a device tensor of leading dimension ld (padding = junk or INF)."""
    rows, cols = host.shape
    ld = ld or ((cols + 7) // 8 * 8)
    fill = I16_INF if junk is None else junk
    t = torch.full((rows, ld), fill, dtype=torch.int16)
    t[:, :cols] = torch.from_numpy(np.ascontiguousarray(host))
    return t.cuda()


# ---------------------------------------------------------------- a1: state enumerator

@pytest.mark.parametrize("m", list(range(1, 12)))
def test_enumerate_states(rd, torch_mod, orc, m):
    torch = torch_mod
    n = rd.state_count(m)
    codes = torch.empty(n, dtype=torch.int32, device="cuda")
    wts = torch.empty(n, dtype=torch.uint8, device="cuda")
    rd.enumerate_states(m, codes, wts)
    ocode, owt = orc.words(m)
    assert np.array_equal(codes.cpu().numpy().view(np.uint32), ocode)
    assert np.array_equal(wts.cpu().numpy().astype(np.int32), owt)


# ---------------------------------------------------------------- a2: transfer matrix

@pytest.mark.parametrize("m", list(range(1, 9)))
def test_transfer_matrix(rd, torch_mod, orc, m):
    A, n = rd.transfer_matrix(m)
    got = A.cpu().numpy()
    assert np.array_equal(got[:, :n], to_i16(orc.transfer(m)))
    assert np.all(got[:, n:] == I16_INF)


def test_transfer_matrix_m9_rows(rd, orc):
    A, n = rd.transfer_matrix(9)
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, 28)]))
    got = A[rows.tolist()].cpu().numpy()
    assert np.array_equal(got[:, :n], to_i16(orc.transfer_rows(9, rows)))


# ---------------------------------------------------------------- a3: (min,+) GEMM

SHAPES = [(1, 1, 1), (7, 9, 5), (33, 33, 33), (128, 256, 32), (129, 257, 33), (300, 520, 700), (1, 777, 640),
          (640, 8, 1000), (1000, 1000, 1000),
          # few output tiles and a long K: the split-K cluster form (8 and 4 slices, ragged last slice)
          (257, 300, 1500), (130, 260, 1030)]


@pytest.mark.parametrize("dist", ["u32", "wide", "dense"])
@pytest.mark.parametrize("shape", SHAPES)
def test_minplus_gemm(rd, torch_mod, orc, shape, dist):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    M, N, K = shape
    a = inputs.matrix(M, K, seed=11, dist=dist)
    b = inputs.matrix(K, N, seed=12, dist=dist)
    # padding columns hold junk that a correct kernel never reads
    A = upload(torch, a, ld=(K + 7) // 8 * 8 + 8, junk=-7)
    B = upload(torch, b, ld=(N + 7) // 8 * 8 + 16, junk=-7)
    C = torch.full((M, (N + 7) // 8 * 8), 12345, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.minplus_gemm(A, B, C, M, N, K, min_out=mn)
    want = orc.minplus_i16(a, b)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :N].astype(np.int32), want)
    assert np.all(got[:, N:] == 12345)  # nothing written past column N
    assert mn.item() == want.min()


# stream-K: one tile over 7 k-tiles (7 CTAs of one unit each), 9 tiles of 63 k-tiles over 1-2 units per CTA,
# 128 tiles of 2 k-tiles (every tile split in two), and ragged M, N, K in every position
SK_SHAPES = SHAPES + [(128, 256, 224), (384, 768, 2000), (2048, 2048, 64), (1024, 1024, 1024), (640, 1100, 3001)]


@pytest.mark.parametrize("shape", SK_SHAPES)
def test_minplus_gemm_streamk(rd, torch_mod, orc, shape):
    """rd_minplus_gemm_streamk element by element against the oracle, with junk in the padding; the
    workspace's counters are zero again after the call."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    M, N, K = shape
    a = inputs.matrix(M, K, seed=21, dist="u32")
    b = inputs.matrix(K, N, seed=22, dist="u32")
    A = upload(torch, a, ld=(K + 7) // 8 * 8 + 8, junk=-7)
    B = upload(torch, b, ld=(N + 7) // 8 * 8 + 16, junk=-7)
    C = torch.full((M, (N + 7) // 8 * 8), 12345, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = rd.minplus_gemm_streamk_workspace(M, N, K)
    rd.minplus_gemm_streamk(A, B, C, work, M, N, K, min_out=mn)
    want = orc.minplus_i16(a, b)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :N].astype(np.int32), want)
    assert np.all(got[:, N:] == 12345)
    assert mn.item() == want.min()
    tiles = ((M + 127) // 128) * ((N + 255) // 256)
    cnt0 = work.numel() - (4 * tiles + 255) // 256 * 256  # the counters follow the partial tiles
    assert int(work[cnt0:cnt0 + 4 * tiles].view(torch.int32).abs().sum().item()) == 0


@pytest.mark.parametrize("shape", [(0, 16, 16), (16, 0, 16), (16, 16, 0), (300, 257, 0)])
def test_minplus_gemm_streamk_degenerate(rd, torch_mod, shape):
    """Empty products through the stream-K entry point: no rows or columns writes nothing, no terms (K = 0)
    gives an all-RD_INF C and min_out = RD_INF; the workspace is not touched."""
    torch = torch_mod
    M, N, K = shape
    A = torch.zeros((max(M, 1), max((K + 7) // 8 * 8, 8)), dtype=torch.int16, device="cuda")
    B = torch.zeros((max(K, 1), max((N + 7) // 8 * 8, 8)), dtype=torch.int16, device="cuda")
    C = torch.full((max(M, 1), max((N + 7) // 8 * 8, 8)), 77, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = rd.minplus_gemm_streamk_workspace(max(M, 1), max(N, 1), max(K, 1))
    rd.minplus_gemm_streamk(A, B, C, work, M, N, K, min_out=mn)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    if M > 0 and N > 0:
        assert np.all(got[:M, :N] == I16_INF)
    else:
        assert np.all(got == 77)
    assert mn.item() == int(I16_INF)
    assert int(work.sum().item()) == 0


def test_minplus_gemm_streamk_reuses_its_workspace(rd, torch_mod, orc):
    """One workspace through products of different shapes on two streams in turn (each call after the
    previous one), then a short workspace and a misaligned one are refused."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    shapes = [(1024, 1024, 1024), (257, 300, 1500), (2048, 2048, 64), (129, 257, 33), (1024, 1024, 1024)]
    work = rd.minplus_gemm_streamk_workspace(2048, 2048, 1024)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for i, (M, N, K) in enumerate(shapes):
        a = inputs.matrix(M, K, seed=31 + i, dist="wide")
        b = inputs.matrix(K, N, seed=41 + i, dist="wide")
        A, B = upload(torch, a, ld=(K + 7) // 8 * 8), upload(torch, b, ld=(N + 7) // 8 * 8)
        C = torch.empty((M, (N + 7) // 8 * 8), dtype=torch.int16, device="cuda")
        s = streams[i % 2]
        s.wait_stream(torch.cuda.current_stream())
        rd.minplus_gemm_streamk(A, B, C, work, M, N, K, stream=s)
        s.synchronize()
        assert np.array_equal(C.cpu().numpy()[:, :N].astype(np.int32), orc.minplus_i16(a, b)), (M, N, K)
    A = torch.zeros((256, 256), dtype=torch.int16, device="cuda")
    C = torch.empty_like(A)
    need = rd.minplus_gemm_streamk_work_bytes(256, 256, 256)
    with pytest.raises(rd.RdError) as e:
        rd.minplus_gemm_streamk(A, A, C, work[:need - 256])
    assert e.value.status == rd.RD_ERR_NOMEM
    with pytest.raises(rd.RdError) as e:
        rd.minplus_gemm_streamk(A, A, C, work[16:])
    assert e.value.status == rd.RD_ERR_ARG


@pytest.mark.parametrize("shape", [(1, 300, 1000), (70, 90, 130), (257, 1000, 511), (1030, 129, 2000)])
def test_minplus_gemm_host(rd, torch_mod, orc, shape):
    """The product through the host-buffer entry point: host strides wider than the rows, pinned and
    pageable buffers, two streams in turn with their own staging buffers; element by element."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    M, K, N = shape
    a = inputs.matrix(M, K, seed=81, dist="wide")
    b = inputs.matrix(K, N, seed=82, dist="wide")
    want = orc.minplus_i16(a, b)
    a_wide = np.full((M, K + 5), -1, dtype=np.int16)
    a_wide[:, :K] = a
    b_wide = np.full((K, N + 3), -1, dtype=np.int16)
    b_wide[:, :N] = b
    wbytes = rd.minplus_gemm_host_work_bytes(M, N, K)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    works = [torch.empty(wbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    mins = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in range(2)]
    pinned = [torch.from_numpy(a_wide).pin_memory()[:, :K], torch.from_numpy(b_wide).pin_memory()[:, :N]]
    outs = [torch.full((M, N + 1), 123, dtype=torch.int16).pin_memory()[:, :N] for _ in range(2)]
    for i in range(2):  # pinned, two streams in turn
        rd.minplus_gemm_host(pinned[0], pinned[1], outs[i], works[i], min_out=mins[i], stream=streams[i])
    c_np = np.full((M, N + 2), 321, dtype=np.int16)
    rd.minplus_gemm_host(a_wide[:, :K], b_wide[:, :N], c_np[:, :N], works[0], stream=streams[0])  # pageable
    torch.cuda.synchronize()
    for i in range(2):
        assert np.array_equal(outs[i].numpy().astype(np.int32), want), i
        assert mins[i].item() == want.min()
    assert np.array_equal(c_np[:, :N].astype(np.int32), want)
    assert np.all(c_np[:, N:] == 321)


def test_minplus_gemm_host_rejects_short_work(rd, torch_mod):
    torch = torch_mod
    a = np.zeros((16, 16), dtype=np.int16)
    c = np.zeros((16, 16), dtype=np.int16)
    work = torch.empty(rd.minplus_gemm_host_work_bytes(16, 16, 16) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(rd.RdError) as e:
        rd.minplus_gemm_host(a, a, c, work)
    assert e.value.status == rd.RD_ERR_NOMEM


def test_minplus_gemm_k0_and_empty(rd, torch_mod):
    torch = torch_mod
    A = torch.zeros((5, 8), dtype=torch.int16, device="cuda")
    B = torch.zeros((8, 16), dtype=torch.int16, device="cuda")
    C = torch.zeros((5, 16), dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.minplus_gemm(A, B, C, 5, 16, 0, min_out=mn)
    assert torch.all(C == I16_INF) and mn.item() == I16_INF
    rd.minplus_gemm(A, B, C, 0, 16, 8)  # nothing to do
    rd.minplus_gemm(A, B, C, 5, 0, 8)


def test_minplus_gemm_all_infinite_rows(rd, torch_mod, orc):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    a = inputs.matrix(200, 300, seed=21, dist="wide")
    a[17, :] = I16_INF
    b = inputs.matrix(300, 260, seed=22, dist="wide")
    b[:, 100] = I16_INF
    A, B = upload(torch, a), upload(torch, b)
    C = torch.empty((200, 264), dtype=torch.int16, device="cuda")
    rd.minplus_gemm(A, B, C, 200, 260, 300)
    got = C.cpu().numpy()[:, :260]
    assert np.all(got[17] == I16_INF) and np.all(got[:, 100] == I16_INF)
    assert np.array_equal(got.astype(np.int32), orc.minplus_i16(a, b))


@pytest.mark.parametrize("n", [4096, 16384])
def test_minplus_gemm_full_size_sampled(rd, torch_mod, orc, n):
    """Bench-size operands, 64 sampled entries (plus one full row and column) against the oracle."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    for dist, seeds in (("wide", (31, 32)), ("u32", (1, 2))):
        A = inputs.matrix_torch(n, n, seed=seeds[0], dist=dist, device="cuda")
        B = inputs.matrix_torch(n, n, seed=seeds[1], dist=dist, device="cuda")
        a, b = A.cpu().numpy(), B.cpu().numpy()
        assert np.array_equal(a[:3], inputs.matrix(3, n, seed=seeds[0], dist=dist))
        C = torch.empty((n, n), dtype=torch.int16, device="cuda")
        rd.minplus_gemm(A, B, C)
        rng = np.random.default_rng(n)
        ri, cj = rng.integers(0, n, 64), rng.integers(0, n, 64)
        got = C.cpu().numpy()
        assert np.array_equal(got[ri, cj].astype(np.int32), orc.minplus_i16_entries(a, b, ri, cj))
        r0 = int(rng.integers(0, n))
        assert np.array_equal(got[r0].astype(np.int32), orc.minplus_i16(a[r0:r0 + 1], b)[0])
        del A, B, C


# ---------------------------------------------------------------- a4-a6: power driver

def run_power(rd, torch, A, n, kmax, slots):
    work = rd.power_workspace(n, A.stride(0), kmax, slots)
    r = rd.power_until_periodic(A, n, kmax, work)
    return r, work


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7])
def test_power_until_periodic_matches_oracle(rd, torch_mod, orc, m):
    A, n = rd.transfer_matrix(m)
    r, work = run_power(rd, torch_mod, A, n, kmax=48, slots=8)
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
            ok = want[want != INF64]
            assert np.array_equal(pk, to_i16(np.where(want == INF64, INF64, want - ok.min()))), k


def test_power_m8_matches_oracle(rd, torch_mod, orc):
    A, n = rd.transfer_matrix(8)
    r, _ = run_power(rd, torch_mod, A, n, kmax=30, slots=8)
    o = orc.power_until_periodic(8, kmax=30)
    assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"]) == (21, 5, 18)
    assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1])


def test_power_m9_full_size(rd, torch_mod, orc):
    """m = 9 (N = 21909): the oracle's first repeat and gamma[1..j] (its row-streamed search), Table 2's
    triple, the row DP for n <= 7, and sampled rows of the resident powers."""
    A, n = rd.transfer_matrix(9)
    slots = 8
    r, work = run_power(rd, torch_mod, A, n, kmax=40, slots=slots)
    table = {int(x[0]): tuple(map(int, x[1:])) for x in read_golden("paper_table2_periods.txt")}
    assert r["found"] and (r["k"], r["p"], r["q"]) == table[9]
    o = oracle_m9()
    assert (r["k"], r["p"], r["q"], r["j"]) == (o["k"], o["p"], o["q"], o["j"])
    assert [int(x) for x in r["gamma"][1:r["j"] + 1]] == o["gamma"][1:o["j"] + 1]
    g = r["gamma"]
    for nn in range(3, 8):
        assert g[nn] == orc.row_dp(9, nn)
    # rows of the last resident powers equal rows of A^k up to one constant per power
    rng = np.random.default_rng(99)
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 10)]))
    ora = orc.power_rows(9, rows, r["j"])
    ld = A.stride(0)
    for k in range(r["j"] - slots + 1, r["j"] + 1):
        off = rd.power_slot(n, ld, 40, work.numel(), k)
        pk = work[off:off + n * ld * 2].view(torch_mod.int16).view(n, ld)[rows.tolist(), :n].cpu().numpy()
        want = ora[k - 1]
        fin = want != INF64
        assert np.array_equal(pk == I16_INF, ~fin)
        d = want[fin] - pk[fin].astype(np.int64)
        assert np.all(d == d[0]) and pk[fin].min() >= 0, k


def test_power_not_found_within_kmax(rd, torch_mod, orc):
    A, n = rd.transfer_matrix(3)
    r, _ = run_power(rd, torch_mod, A, n, kmax=9, slots=4)
    assert r["status"] == rd.RD_NOT_FOUND and not r["found"]
    assert np.array_equal(r["gamma"][1:10], orc.gamma_direct(3, 9)[1:10])


@pytest.mark.parametrize("m,kmax", [(5, 20), (6, 7)])
def test_power_not_found_within_kmax_step_kernels(rd, torch_mod, orc, m, kmax):
    """The dense search through the step kernels (N > 128, blocks of steps queued ahead of the host's check)
    stopped by kmax before its repeat: RD_NOT_FOUND, gamma[1..kmax] equal to the oracle's, nothing past kmax."""
    A, n = rd.transfer_matrix(m)
    assert n > 128
    r, _ = run_power(rd, torch_mod, A, n, kmax=kmax, slots=8)
    assert r["status"] == rd.RD_NOT_FOUND and not r["found"]
    want = orc.power_until_periodic(m, kmax=kmax)
    assert not want["found"]
    assert np.array_equal(r["gamma"][1:kmax + 1], want["gamma"][1:kmax + 1])


@pytest.mark.parametrize("R", [1, 2])
def test_power_sparse_not_found_within_kmax(rd, torch_mod, orc, R):
    """The dense x sparse search stopped by kmax before its repeat (m = 6, j = 24): RD_NOT_FOUND with
    gamma[1..kmax] equal to the oracle's; the same workspace then finds (19, 5, 14)."""
    A, n = rd.transfer_matrix(6)
    plan = rd.sparse_plan(A, n, n, R)
    work = rd.power_workspace(n, A.stride(0), 48, 8)
    r = rd.power_until_periodic_sparse(A, n, plan, 20, work)
    assert r["status"] == rd.RD_NOT_FOUND and not r["found"]
    want = orc.power_until_periodic(6, kmax=20)
    assert np.array_equal(r["gamma"][1:21], want["gamma"][1:21])
    r2 = rd.power_until_periodic_sparse(A, n, plan, 48, work)
    assert (r2["k"], r2["p"], r2["q"]) == (19, 5, 14)


def test_power_ring_too_short(rd, torch_mod):
    A, n = rd.transfer_matrix(2)  # period 4 needs at least 5 slots
    work = rd.power_workspace(n, A.stride(0), 40, 3)
    with pytest.raises(rd.RdError) as e:
        rd.power_until_periodic(A, n, 40, work)
    assert e.value.status == rd.RD_ERR_NOMEM


def test_power_range_violation(rd, torch_mod):
    torch = torch_mod
    A = torch.full((16, 16), 0x2000, dtype=torch.int16, device="cuda")  # entries above RD_MAX_FINITE
    work = rd.power_workspace(16, 16, 8, 4)
    with pytest.raises(rd.RdError) as e:
        rd.power_until_periodic(A, 16, 8, work)
    assert e.value.status == rd.RD_ERR_RANGE


@pytest.mark.parametrize("n,seed", [(40, 1), (100, 2), (257, 3)])
def test_power_synthetic_matrix(rd, torch_mod, orc, n, seed):
    from paper_2409_17658_gb300 import inputs

    a = inputs.matrix(n, n, seed=seed, dist="u32")
    A = upload(torch_mod, a)
    r, _ = run_power(rd, torch_mod, A, n, kmax=40, slots=41)
    a64 = np.where(a == I16_INF, INF64, a.astype(np.int64))
    o = orc.power_until_periodic(0, a=a64, kmax=40)
    assert r["found"] == o["found"]
    if o["found"]:
        assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"])
    assert np.array_equal(r["gamma"][1:o["j"] + 1], o["gamma"][1:o["j"] + 1])


# ---------------------------------------------------------------- a7: closed-form evaluation

def test_gamma_R_matches_algorithm1(rd, orc):
    for m in range(1, 7):
        direct = orc.gamma_direct(m, 70)
        r = orc.power_until_periodic(m, kmax=48)
        for n in range(3, 71):
            assert rd.gamma_R(m, n) == direct[n], (m, n)
        for n in (100, 1001, 12345):
            assert rd.gamma_R(m, n) == orc.gamma_from_period(r["gamma"], r["k"], r["p"], r["q"], n)
    for n in range(3, 200):
        assert rd.gamma_R(1, n) == math.ceil(2 * n / 3)


def test_gamma_R_m9_closed_form(rd):
    """rd_gamma_R(9, n) against the oracle's gamma for n < k + p and, beyond, the solution of Prop. 7 from the
    oracle's first repeat; and against the m = 9 closed form printed in Sec. 4.C (4n if 5 | n, else 4n + 2)."""
    o = oracle_m9()
    for n in range(3, 501):
        if n < o["k"] + o["p"]:
            want = o["gamma"][n]
        else:
            want = o["gamma"][o["k"] + (n - o["k"]) % o["p"]] + o["q"] * ((n - o["k"]) // o["p"])
        got = rd.gamma_R(9, n)
        assert got == want, n
        assert got == (4 * n if n % 5 == 0 else 4 * n + 2), n


def test_gamma_R_closed_forms_m7(rd):
    for n in range(3, 120):
        want = 20 if n == 6 else math.ceil(16 * n / 5) + (0 if n % 5 == 0 else 1)
        assert rd.gamma_R(7, n) == want, n


# ---------------------------------------------------------------- f1: dense x sparse step

SPARSE_SHAPES = [(1, 1, 1), (5, 9, 13), (33, 33, 33), (37, 300, 1000), (130, 200, 1030), (257, 640, 2049)]


@pytest.mark.parametrize("R", [1, 2, 4, 8])
@pytest.mark.parametrize("shape", SPARSE_SHAPES)
def test_sparse_minplus(rd, torch_mod, orc, shape, R):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    M, K, N = shape
    a = inputs.matrix(M, K, seed=41, dist="wide")
    keep = inputs.matrix(M, K, seed=43, dist="u32") < 3  # about 5 % of the entries stay finite
    a = np.where(keep, a, I16_INF).astype(np.int16)
    b = inputs.matrix(K, N, seed=42, dist="wide")
    A = upload(torch, a, junk=-5)
    B = upload(torch, b, junk=-5)
    plan = rd.sparse_plan(A, M, K, R)
    # the plan lists, per block of R rows, the union of finite columns
    fin = a != I16_INF
    want_entries = sum(int(fin[i0:i0 + R].any(0).sum()) for i0 in range(0, M, R))
    assert plan["entries"] == want_entries
    C = torch.full((M, (N + 7) // 8 * 8), 777, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.sparse_minplus(plan, B, C, N, min_out=mn)
    want = orc.minplus_i16(a, b)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :N].astype(np.int32), want)
    assert np.all(got[:, N:] == 777)
    assert mn.item() == want.min()


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
def test_power_sparse_matches_oracle(rd, torch_mod, orc, m):
    A, n = rd.transfer_matrix(m)
    plan = rd.sparse_plan(A, n, n, 4)
    work = rd.power_workspace(n, A.stride(0), 40, 8)
    r = rd.power_until_periodic_sparse(A, n, plan, 40, work)
    o = orc.power_until_periodic(m, kmax=40)
    assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"])
    assert np.array_equal(r["gamma"][1:r["j"] + 1], o["gamma"][1:o["j"] + 1])


@pytest.mark.parametrize("R", [1, 2, 8])
def test_power_sparse_m9_equals_dense(rd, torch_mod, orc, R):
    A, n = rd.transfer_matrix(9)
    plan = rd.sparse_plan(A, n, n, R)
    work = rd.power_workspace(n, A.stride(0), 40, 8)
    r = rd.power_until_periodic_sparse(A, n, plan, 40, work)
    o = oracle_m9()
    assert (r["k"], r["p"], r["q"], r["j"]) == (o["k"], o["p"], o["q"], o["j"]) == (22, 5, 20, 27)
    assert [int(x) for x in r["gamma"][1:r["j"] + 1]] == o["gamma"][1:o["j"] + 1]
    for nn in range(3, 8):
        assert r["gamma"][nn] == orc.row_dp(9, nn)
    # same gamma sequence as the dense step
    work2 = rd.power_workspace(n, A.stride(0), 40, 8)
    d = rd.power_until_periodic(A, n, 40, work2)
    assert np.array_equal(r["gamma"], d["gamma"])
    # the resident final power agrees with the dense run bit for bit
    off = rd.power_slot(n, A.stride(0), 40, work.numel(), r["j"])
    off2 = rd.power_slot(n, A.stride(0), 40, work2.numel(), d["j"])
    ld = A.stride(0)
    assert torch_mod.equal(work[off:off + n * ld * 2].view(torch_mod.int16).view(n, ld)[:, :n],
                           work2[off2:off2 + n * ld * 2].view(torch_mod.int16).view(n, ld)[:, :n])


# ---------------------------------------------------------------- f3: m = 10 (N = 64769)

def test_power_m10(rd, torch_mod, orc):
    """m = 10 has no Table 2 row.  The oracle's stored first repeat and gamma[1..j] (its row-streamed search)
    are compared exactly.  What the paper fixes: gamma = 22n/5 for n = 0 mod 5, n >= 10
    (Cor. 12) and n = 5 (Remark 13), gamma >= ceil(22n/5) for n >= 10 (Theorem 11); the path
    DP gives n <= 7; sampled rows of the resident powers are checked against the oracle."""
    torch = torch_mod
    m = 10
    A, n = rd.transfer_matrix(m)
    assert n == 64769
    ld = A.stride(0)
    kmax = 48
    work = rd.power_workspace(n, ld, kmax, 8)
    plan = rd.sparse_plan(A, n, n, 2)
    r = rd.power_until_periodic_sparse(A, n, plan, kmax, work)
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
    rng = np.random.default_rng(10)
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
    assert rd.gamma_R(m, 100) == 440 and rd.gamma_R(m, 7) == orc.row_dp(m, 7)


# ---------------------------------------------------------------- f2: Appendix loss variant

@pytest.mark.parametrize("m", [2, 3, 4, 5, 6])
def test_transfer_loss_matrix(rd, torch_mod, orc, m):
    torch = torch_mod
    n = rd.state_count(m)
    A = torch.empty((n, rd.padded_dim(n)), dtype=torch.int16, device="cuda")
    rd.build_transfer_loss(m, A)
    want = orc.transfer_loss(m)
    shifted = np.where(want == INF64, INF64, want + rd.loss_shift(m))
    got = A.cpu().numpy()
    assert np.array_equal(got[:, :n], to_i16(shifted))
    assert np.all(got[:, n:] == I16_INF)


@pytest.mark.parametrize("m", [4, 5, 6])
@pytest.mark.parametrize("sparse", [False, True])
def test_loss_variant_power(rd, torch_mod, orc, m, sparse):
    torch = torch_mod
    n = rd.state_count(m)
    A = torch.empty((n, rd.padded_dim(n)), dtype=torch.int16, device="cuda")
    rd.build_transfer_loss(m, A)
    work = rd.power_workspace(n, A.stride(0), 48, 8)
    if sparse:
        r = rd.power_until_periodic_sparse(A, n, rd.sparse_plan(A, n, n, 2), 48, work)
    else:
        r = rd.power_until_periodic(A, n, 48, work)
    s = rd.loss_shift(m)
    o = orc.power_until_periodic(0, a=orc.transfer_loss(m), kmax=48)
    assert r["found"] and o["found"]
    assert (r["k"], r["p"], r["q"] - s * r["p"]) == (o["k"], o["p"], o["q"])
    j = r["j"]
    assert np.array_equal(r["gamma"][1:j + 1] - s * np.arange(1, j + 1), o["gamma"][1:j + 1])
    if m == 4:
        assert (r["k"], r["p"], r["q"] - s * r["p"]) == (30, 1, 1)  # the Appendix's relation


# ---------------------------------------------------------------- batched products (one persistent launch)

def test_minplus_gemm_batched(rd, torch_mod, orc):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    rng = np.random.default_rng(77)
    shapes = [(int(rng.integers(1, 400)), int(rng.integers(1, 600)), int(rng.integers(1, 500))) for _ in range(24)]
    shapes += [(0, 16, 16), (16, 16, 0), (300, 257, 129)]
    probs, want = [], []
    for i, (M, N, K) in enumerate(shapes):
        dist = ("wide", "u32", "dense")[i % 3]
        a = inputs.matrix(M, K, seed=100 + i, dist=dist) if M and K else np.zeros((M, K), np.int16)
        b = inputs.matrix(K, N, seed=200 + i, dist=dist) if K and N else np.zeros((K, N), np.int16)
        A = upload(torch, a, junk=-3) if M and K else torch.zeros((max(M, 1), 8), dtype=torch.int16, device="cuda")
        B = upload(torch, b, junk=-3) if K and N else torch.zeros((max(K, 1), (N + 7) // 8 * 8 or 8),
                                                                 dtype=torch.int16, device="cuda")
        C = torch.full((max(M, 1), (N + 7) // 8 * 8), 555, dtype=torch.int16, device="cuda")
        mn = torch.zeros(1, dtype=torch.int32, device="cuda")
        probs.append((A, B, C, M, N, K, mn))
        if M and N:
            w = orc.minplus_i16(a, b) if K else np.full((M, N), I16_INF, np.int32)
        else:
            w = None
        want.append(w)
    rd.minplus_gemm_batched(probs)
    torch.cuda.synchronize()
    for (A, B, C, M, N, K, mn), w in zip(probs, want):
        if w is None:
            assert torch.all(C == 555)
            continue
        got = C.cpu().numpy()
        assert np.array_equal(got[:M, :N].astype(np.int32), w), (M, N, K)
        assert np.all(got[:M, N:] == 555)
        assert mn.item() == w.min()


# ---------------------------------------------------------------- several searches advanced together

@pytest.mark.parametrize("graph_steps", [0, 8])
def test_power_multi_equals_single_runs(rd, torch_mod, orc, graph_steps):
    torch = torch_mod
    kmax = 48
    runs, singles = [], []
    for m in range(1, 10):
        A, n = rd.transfer_matrix(m)
        plan = rd.sparse_plan(A, n, n, 2)
        runs.append((A, n, plan, rd.power_workspace(n, A.stride(0), kmax, 8)))
    res = rd.power_until_periodic_multi(runs, 2, kmax, graph_steps=graph_steps)
    for m, (A, n, plan, _), r in zip(range(1, 10), runs, res):
        alone = rd.power_until_periodic_sparse(A, n, plan, kmax, rd.power_workspace(n, A.stride(0), kmax, 8))
        assert (r["k"], r["p"], r["q"]) == (alone["k"], alone["p"], alone["q"]), m
        assert np.array_equal(r["gamma"], alone["gamma"]), m
        if m <= 7:
            o = orc.power_until_periodic(m, kmax=kmax)
            assert (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"]), m
    assert (res[8]["k"], res[8]["p"], res[8]["q"]) == (22, 5, 20)


@pytest.mark.parametrize("graph_steps", [0, 8])
def test_power_multi_mixed_found_and_not_found(rd, torch_mod, orc, graph_steps):
    """kmax = 15 lets m = 1..3 find their repeats (j = 9, 10, 15) while m = 4..8 run out: each run's status, and its
    relation and gamma up to j (found) or kmax (not found), equal the oracle's; m = 8 runs with the row split."""
    kmax = 15
    runs = []
    for m in range(1, 9):
        A, n = rd.transfer_matrix(m)
        plan = rd.split_plan(m, x_ld=A.stride(0)) if m == 8 else rd.sparse_plan(A, n, n, 2)
        runs.append((A, n, plan, rd.power_workspace(n, A.stride(0), kmax, 8)))
    res = rd.power_until_periodic_multi(runs, 2, kmax, graph_steps=graph_steps)
    for m, r in zip(range(1, 9), res):
        o = orc.power_until_periodic(m, kmax=kmax) if m <= 7 else None
        if m == 8:
            assert r["status"] == rd.RD_NOT_FOUND
            continue
        assert r["found"] == o["found"], m
        if o["found"]:
            assert r["status"] == rd.RD_OK and (r["k"], r["p"], r["q"]) == (o["k"], o["p"], o["q"]), m
        else:
            assert r["status"] == rd.RD_NOT_FOUND, m
        assert np.array_equal(r["gamma"][1:o["j"] + 1], o["gamma"][1:o["j"] + 1]), m


def test_power_multi_wait_runs_out(rd, torch_mod, orc):
    """The one-launch step's bounded wait gives up and says so, and the GPU stays usable.  The run of m = 5 is
    stalled: its product level counts one item more than it has, as a lost item would, so its normaliser
    items wait until the bound (50 ms) runs out.  That run stops with RD_ERR_TIMEOUT; the other runs' relations
    and gamma equal the oracle's; the next call without a stall is exact for every run."""
    kmax = 48
    ms = (3, 4, 5, 6, 7)
    runs = []
    for m in ms:
        A, n = rd.transfer_matrix(m)
        runs.append((A, n, rd.sparse_plan(A, n, n, 2), rd.power_workspace(n, A.stride(0), kmax, 8)))
    want = {m: orc.power_until_periodic(m, kmax=kmax) for m in ms}
    res = rd.power_until_periodic_multi(runs, 2, kmax, graph_steps=8, wait_ms=50, stall_run=2)
    assert res[2]["status"] == rd.RD_ERR_TIMEOUT
    for i, m in enumerate(ms):
        if i == 2:
            continue
        o = want[m]
        assert (res[i]["k"], res[i]["p"], res[i]["q"]) == (o["k"], o["p"], o["q"]), m
        assert np.array_equal(res[i]["gamma"][1:o["j"] + 1], o["gamma"][1:o["j"] + 1]), m
    res = rd.power_until_periodic_multi(runs, 2, kmax, graph_steps=8)
    for i, m in enumerate(ms):
        o = want[m]
        assert (res[i]["k"], res[i]["p"], res[i]["q"]) == (o["k"], o["p"], o["q"]), m
        assert np.array_equal(res[i]["gamma"][1:o["j"] + 1], o["gamma"][1:o["j"] + 1]), m


def test_power_multi_bounded_rejects_bad_knobs(rd, torch_mod):
    lib = rd._lib()
    arr = (rd.PowerRun * 1)()
    assert lib.rd_power_until_periodic_multi_bounded(arr, 1, 2, 8, 0, 0, -1, None) == rd.RD_ERR_ARG
    assert lib.rd_power_until_periodic_multi_bounded(arr, 1, 2, 8, 0, 100, 1, None) == rd.RD_ERR_ARG
    assert lib.rd_power_until_periodic_multi_bounded(arr, 1, 2, 8, 0, 100, -2, None) == rd.RD_ERR_ARG


@pytest.mark.parametrize("R", [1, 2, 4, 8])
@pytest.mark.parametrize("shape", SPARSE_SHAPES + [(300, 2000, 2500)])
def test_sparse_minplus_tma(rd, torch_mod, orc, shape, R):
    """The bulk-copy (cp.async.bulk + mbarrier ring) product, ragged slabs included."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    M, K, N = shape
    a = inputs.matrix(M, K, seed=51, dist="wide")
    keep = inputs.matrix(M, K, seed=53, dist="u32") < 3
    a = np.where(keep, a, I16_INF).astype(np.int16)
    b = inputs.matrix(K, N, seed=52, dist="wide")
    A = upload(torch, a, junk=-5)
    B = upload(torch, b, junk=-5)
    plan = rd.sparse_plan(A, M, K, R)
    C = torch.full((M, (N + 7) // 8 * 8), 777, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.sparse_minplus_tma(plan, B, C, err, N, min_out=mn)
    assert err.item() == 0
    want = orc.minplus_i16(a, b)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :N].astype(np.int32), want)
    assert np.all(got[:, N:] == 777)
    assert mn.item() == want.min()


@pytest.mark.parametrize("R", [1, 8])
def test_sparse_minplus_tma_wait_runs_out(rd, torch_mod, orc, R):
    """The bulk-copy kernel's bounded wait gives up and says so, and the GPU stays usable.  Every CTA's
    producer stops before entry 3 of its block, as a lost copy would; the consumers wait for that entry,
    give up after 4096 try_wait rounds with no copy in flight, and report the timeout bit (8).  The next
    call, with the default limit and no stop, is bit-exact against the oracle."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    M, K, N = 130, 200, 1030
    a = inputs.matrix(M, K, seed=71, dist="wide")
    keep = inputs.matrix(M, K, seed=73, dist="u32") < 6
    a = np.where(keep, a, I16_INF).astype(np.int16)
    b = inputs.matrix(K, N, seed=72, dist="wide")
    A = upload(torch, a)
    B = upload(torch, b)
    plan = rd.sparse_plan(A, M, K, R)
    starts = plan["block_start"].cpu().numpy()
    assert (np.diff(starts) > 3).any()  # some blocks need the withheld entry
    C = torch.full((M, (N + 7) // 8 * 8), 777, dtype=torch.int16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.sparse_minplus_tma_bounded(plan, B, C, err, wait_limit=4096, stop_at=3, N=N)
    torch.cuda.synchronize()
    assert err.item() == 8
    err.zero_()
    rd.sparse_minplus_tma_bounded(plan, B, C, err, wait_limit=1 << 20, stop_at=-1, N=N)
    assert err.item() == 0
    assert np.array_equal(C.cpu().numpy()[:, :N].astype(np.int32), orc.minplus_i16(a, b))


def test_sparse_minplus_tma_bounded_rejects_bad_knobs(rd, torch_mod):
    lib = rd._lib()
    import ctypes

    vp = ctypes.c_void_p
    err = torch_mod.zeros(1, dtype=torch_mod.int32, device="cuda")
    e = vp(err.data_ptr())
    assert lib.rd_sparse_minplus_tma_bounded(1, 0, None, None, None, 8, 0, None, 8, None, e, 0, -1, None) == rd.RD_ERR_ARG
    assert lib.rd_sparse_minplus_tma_bounded(1, 0, None, None, None, 8, 0, None, 8, None, e, 16, -2, None) == rd.RD_ERR_ARG
    assert lib.rd_sparse_minplus_tma_bounded(1, 0, None, None, None, 8, 0, None, 8, None, e, 16, -1, None) == rd.RD_OK


# ---------------------------------------------------------------- vector x matrix (one row against an N x N operand)

@pytest.mark.parametrize("K,N", [(1, 1), (5, 13), (300, 1000), (9000, 777), (8192, 264), (20000, 2049)])
def test_minplus_gemv(rd, torch_mod, orc, K, N):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    x = inputs.matrix(1, K, seed=61, dist="wide")
    b = inputs.matrix(K, N, seed=62, dist="wide")
    X = torch.from_numpy(x[0].copy()).cuda()
    B = upload(torch, b, junk=-9)
    y = torch.full(((N + 7) // 8 * 8,), 4444, dtype=torch.int16, device="cuda")
    mn = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd.minplus_gemv(X, B, y, N, K, min_out=mn)
    want = orc.minplus_i16(x, b)[0]
    got = y.cpu().numpy()
    assert np.array_equal(got[:N].astype(np.int32), want)
    assert np.all(got[N:] == 4444)
    assert mn.item() == want.min()
    # the same through rd_minplus_gemm with M = 1
    A = upload(torch, x)
    C = torch.empty((1, (N + 7) // 8 * 8), dtype=torch.int16, device="cuda")
    rd.minplus_gemm(A, B, C, 1, N, K, min_out=mn)
    assert np.array_equal(C.cpu().numpy()[0, :N].astype(np.int32), want) and mn.item() == want.min()


def test_minplus_gemv_full_size(rd, torch_mod, orc):
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    n = 16384
    B = inputs.matrix_torch(n, n, seed=2, device="cuda")
    x = inputs.matrix(1, n, seed=1)
    y = torch.empty(n, dtype=torch.int16, device="cuda")
    rd.minplus_gemv(torch.from_numpy(x[0].copy()).cuda(), B, y)
    assert np.array_equal(y.cpu().numpy().astype(np.int32), orc.minplus_i16(x, B.cpu().numpy())[0])


def test_minplus_gemm_n32768_sampled(rd, torch_mod, orc):
    """The largest size of the synthetic sweep: 64 sampled entries against the oracle."""
    torch = torch_mod
    from paper_2409_17658_gb300 import inputs

    n = 32768
    A = inputs.matrix_torch(n, n, seed=71, dist="wide", device="cuda")
    B = inputs.matrix_torch(n, n, seed=72, dist="wide", device="cuda")
    C = torch.empty((n, n), dtype=torch.int16, device="cuda")
    rd.minplus_gemm(A, B, C)
    rng = np.random.default_rng(n)
    ri, cj = rng.integers(0, n, 64), rng.integers(0, n, 64)
    a_rows = A[torch.from_numpy(ri).cuda()].cpu().numpy()
    b_cols = B[:, torch.from_numpy(cj).cuda()].cpu().numpy()
    want = np.array([orc.minplus_i16(a_rows[e:e + 1], b_cols[:, e:e + 1])[0, 0] for e in range(64)])
    assert np.array_equal(C[torch.from_numpy(ri).cuda(), torch.from_numpy(cj).cuda()].cpu().numpy().astype(np.int32),
                          want)
