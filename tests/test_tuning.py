"""The tuning table: host-only entry points (rd_tune_set / get / lookup / bucket) and its JSON file.

No GPU is needed: the table lives on the host, and nothing here launches a kernel.
"""
import json

import pytest


@pytest.fixture(scope="module")
def rd():
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    return rd


@pytest.fixture(autouse=True)
def empty_table(rd):
    rd.tune_set([])
    yield
    rd.tune_set([])


def test_bucket_is_ceil_log2(rd):
    for x, b in [(0, 0), (1, 0), (2, 1), (3, 2), (4, 2), (5, 3), (1024, 10), (1025, 11), (64769, 16), (1 << 40, 40)]:
        assert rd.tune_bucket(x) == b, x


def test_set_get_lookup_round_trip(rd):
    entries = [dict(mode="gemm_splitk", key=10, aux=10, p=[8, 0, 0, 0], ms=0.05),
               dict(mode="split", key=9, aux=4, p=[64, 8, 128, 4], ms=1.5),
               dict(mode="sparse_r", key=15, aux=0, p=[2, 0, 0, 0], ms=4.75)]
    rd.tune_set(entries)
    assert rd.tune_table() == entries
    assert rd.tune_lookup(rd.RD_TUNE_SPLIT, 9, 4) == entries[1]
    assert rd.tune_lookup(rd.RD_TUNE_SPLIT, 9, 5) is None
    assert rd.tune_lookup(rd.RD_TUNE_GEMM_SPLITK, 10, 10)["p"][0] == 8
    rd.tune_set([])
    assert rd.tune_table() == []


@pytest.mark.parametrize("bad", [
    dict(mode=9, key=1, aux=0, p=[1]),                       # unknown mode
    dict(mode="gemm_splitk", key=10, aux=10, p=[3]),         # S not in {1, 2, 4, 8}
    dict(mode="gemm_splitk", key=10, aux=10, p=[16]),
    dict(mode="gemm_splitk", key=10, aux=10, p=[2, 2]),        # tile 0 or 1
    dict(mode="split", key=9, aux=9, p=[64, 8, 64, 8]),      # j must be < m
    dict(mode="split", key=1, aux=0, p=[64, 8, 64, 8]),      # m >= 2
    dict(mode="split", key=9, aux=4, p=[96, 8, 64, 8]),      # width not 32, 64, 128 or 256
    dict(mode="split", key=9, aux=4, p=[64, 0, 64, 8]),      # slabs per CTA in 1..64
    dict(mode="split", key=9, aux=4, p=[64, 8, 64, 65]),
    dict(mode="sparse_r", key=15, aux=1, p=[2]),             # aux must be 0
    dict(mode="sparse_r", key=15, aux=0, p=[5]),
])
def test_set_refuses_bad_entries_and_keeps_the_table(rd, bad):
    good = [dict(mode="gemm_splitk", key=12, aux=12, p=[1, 0, 0, 0], ms=2.2)]
    rd.tune_set(good)
    with pytest.raises(rd.RdError):
        rd.tune_set(good + [bad])
    assert rd.tune_table() == good


def test_set_refuses_duplicate_keys_and_overflow(rd):
    e = dict(mode="gemm_splitk", key=10, aux=10, p=[2, 0, 0, 0], ms=-1.0)
    with pytest.raises(rd.RdError):
        rd.tune_set([e, dict(e, p=[4, 0, 0, 0])])
    many = [dict(mode="gemm_splitk", key=k % 64, aux=k // 64, p=[1, 0, 0, 0], ms=-1.0) for k in range(rd.RD_TUNE_MAX)]
    rd.tune_set(many)
    assert len(rd.tune_table()) == rd.RD_TUNE_MAX
    with pytest.raises(rd.RdError):
        rd.tune_set(many + [dict(mode="sparse_r", key=1, aux=0, p=[1, 0, 0, 0], ms=-1.0)])
    assert len(rd.tune_table()) == rd.RD_TUNE_MAX


def test_json_save_load(rd, tmp_path):
    from paper_2409_17658_gb300 import tuning

    entries = [dict(mode="gemm_splitk", key=11, aux=11, p=[2, 0, 0, 0], ms=0.295),
               dict(mode="split", key=10, aux=5, p=[128, 4, 64, 16], ms=14.6)]
    rd.tune_set(entries)
    path = str(tmp_path / "tune.json")
    doc = tuning.save(path, device="GPU-A")
    assert doc["format"] == tuning.FORMAT and json.load(open(path)) == doc
    rd.tune_set([])
    assert tuning.load(path, device="GPU-B") == 0 and rd.tune_table() == []  # another device's table
    assert tuning.load(path, device="GPU-A") == 2 and rd.tune_table() == entries
    # merge: a current entry with another key stays, one with the same key is replaced by the file's
    mine = [dict(mode="sparse_r", key=15, aux=0, p=[1, 0, 0, 0], ms=-1.0),
            dict(mode="split", key=10, aux=5, p=[32, 1, 32, 1], ms=99.0)]
    rd.tune_set(mine)
    tuning.load(path, device="GPU-A")
    got = rd.tune_table()
    assert mine[0] in got and entries[0] in got and entries[1] in got and mine[1] not in got
    tuning.load(path, device="GPU-A", merge=False)
    assert rd.tune_table() == entries
    bad = tmp_path / "bad.json"
    bad.write_text(json.dumps({"format": "other", "entries": []}))
    with pytest.raises(ValueError):
        tuning.load(str(bad), device="GPU-A")
