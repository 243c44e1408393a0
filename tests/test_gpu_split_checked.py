"""The row-split tests again, under the checked build of the library.

compute-sanitizer cannot run on these GPUs, so the library has a build whose row-split passes test every
index they take from plan data and record violations instead of faulting (rd_split_check_flags).  This
test builds it (build.build(checked=True), librd_checked.so) and runs tests/test_gpu_split.py in a child
process that uses it: every row-split parity test must pass with no check firing, and the two cases of
tests/checked_split_cases.py (collected only there) show that the checks fire on rows past an understated
x_rows and that the unstaged pass kernel is clean.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_suite_under_the_checked_build():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    from paper_2409_17658_gb300 import build

    lib = build.build(checked=True)
    torch.cuda.empty_cache()  # leave the child the device memory this process no longer uses
    env = dict(os.environ, RD_CHECKED_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_split.py"),
                        os.path.join(ROOT, "tests", "checked_split_cases.py"), "-m", "gpu", "-x", "-q", "-p",
                        "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "skipped" not in r.stdout, tail
