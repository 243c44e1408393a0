import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden(name):
    """Whitespace-separated rows of a golden file, '#' lines skipped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def oracle_first_repeat(m):
    """The oracle's stored result for m (tests/golden/oracle_m<m>_first_repeat.txt, written by
    tests/golden/make_oracle_first_repeat.py, which calls only the oracle): dict(k, p, q, j, gamma) with
    gamma[n] for n = 1..len - 1."""
    rows = read_golden(f"oracle_m{m}_first_repeat.txt")
    mm, k, p, q, j = map(int, rows[0])
    assert mm == m
    gamma = [None] * (len(rows))
    for n, g in rows[1:]:
        gamma[int(n)] = int(g)
    return dict(k=k, p=p, q=q, j=j, gamma=gamma)


def oracle_m9():
    return oracle_first_repeat(9)


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle
