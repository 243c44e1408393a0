"""Cases that only make sense under the checked build of the library (librd_checked.so, -DRD_CHECKED).

Not collected by a plain `pytest tests` (the file name does not start with test_): test_gpu_split_checked.py
runs this file, with tests/test_gpu_split.py, in a child process whose binding uses the checked build.
"""
import os

import numpy as np
import pytest

from test_gpu_split import I16_INF, INF64, no_index_violations, rd, to_i16, torch_mod  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def needs_checked_build():
    if not os.environ.get("RD_CHECKED_LIB"):
        pytest.fail("run by test_gpu_split_checked.py under the checked build")


def test_checked_build_flags_rows_past_x_rows(rd, torch_mod, orc):
    """The checks fire: with info.x_rows understated by 100, pass 1's outputs and pass 2's inputs past it
    are flagged (bits 8 and 1) and skipped.  X keeps its true size, so those rows stay inside its
    allocation and even an unchecked run would be memory-safe.  With the true x_rows nothing is flagged,
    and the product equals the oracle's."""
    torch = torch_mod
    m = 7
    A, n = rd.transfer_matrix(m)
    plan = rd.split_plan(m, x_ld=A.stride(0))
    info = plan["info"]
    true_rows = info.x_rows
    C = torch.empty_like(A)
    info.x_rows = true_rows - 100
    rd.split_minplus(plan, A, C)
    torch.cuda.synchronize()
    flags = rd.split_check_flags(reset=True)
    assert flags & 1 and flags & 8 and not flags & 6, flags
    info.x_rows = true_rows
    rd.split_minplus(plan, A, C)
    torch.cuda.synchronize()
    assert rd.split_check_flags(reset=True) == 0
    a64 = orc.transfer(m)
    want = to_i16(orc.power_step(a64, a64))
    assert np.array_equal(C[:, :n].cpu().numpy(), want)


def test_checked_build_unstaged_pass(rd, torch_mod, orc):
    """m = 9 with 256-column slabs in pass 2: 368 staged rows of 512 bytes exceed the 64 KB the staged lists
    can address, so pass 2 runs the unstaged kernel (lists read from global memory, slot numbers checked in
    the fold).  No check fires and the product equals the default shape's and, on sampled rows, the oracle's."""
    torch = torch_mod
    m = 9
    A, n = rd.transfer_matrix(m)
    plan = rd.split_plan(m, x_ld=A.stride(0))
    C1 = torch.empty_like(A)
    rd.split_minplus(plan, A, C1)
    plan["info"].w2 = 256
    C2 = torch.empty_like(A)
    rd.split_minplus(plan, A, C2)
    torch.cuda.synchronize()
    assert rd.split_check_flags(reset=True) == 0
    assert torch.equal(C1[:, :n], C2[:, :n])
    rows = np.array([0, 1, n // 2, n - 1])
    want = orc.power_rows(m, rows, 2)[1]
    got = C2[rows.tolist(), :n].cpu().numpy().astype(np.int64)
    assert np.array_equal(np.where(got == I16_INF, INF64, got), want)
