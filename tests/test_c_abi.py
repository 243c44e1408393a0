"""The C ABI from C: tests/c_abi/abi_host.c includes include/rd.h, compiles as C11 with gcc (-pedantic; CUDA's own runtime header needs C11), links against
librd.so and calls the host-side entry points (no GPU needed).  The m = 1 relation record it installs is the
oracle's first repeat, passed on its command line."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_17658_gb300 import build

    return build.build()


def test_header_compiles_as_c_and_links(lib, orc, tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    exe = str(tmp_path / "abi_host")
    build_dir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", f"-I{os.path.join(ROOT, 'include')}",
                    f"-I{cuda_inc}", os.path.join(ROOT, "tests", "c_abi", "abi_host.c"), "-o", exe, f"-L{build_dir}",
                    "-lrd", f"-Wl,-rpath,{build_dir}"], check=True, capture_output=True, text=True)
    r = orc.power_until_periodic(1, kmax=32)
    assert r["found"]
    args = [str(r["k"]), str(r["p"]), str(r["q"]), str(r["j"])] + [str(int(x)) for x in r["gamma"][1:r["j"] + 1]]
    out = subprocess.run([exe, *args], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "FAIL" not in out.stdout and out.stdout.count("ok ") == 12, out.stdout
