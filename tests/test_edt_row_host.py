"""The row pass of the Eq. (1) distance transform on the CPU.

csrc/edt_row.cuh holds the per-thread steps of edt_row_kernel as plain
functions (device functions under nvcc, inline functions under a host
compiler). tests/host/edt_row_host.cpp compiles them with g++ and runs them in
the kernel's order, thread by thread, on random rows with 2 to 256 bands:
sparse, dense, huge and tied distances and staircases of equal g. Every
squared distance must equal a brute-force minimum over all sites, and no
index may leave its array. No GPU and no oracle: the reference is the
definition d2(x) = min over sites q of (x - q)^2 + g(q)^2."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "edt_row_host.cpp")
CSRC = os.path.join(ROOT, "paper_2006_01201_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    out = str(tmp_path_factory.mktemp("edt") / "edt_row_host")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", out, SRC], check=True)
    return out


def test_row_pass_matches_brute_force(exe):
    r = subprocess.run([exe, "1500"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "rows 1500 bad 0 oob 0"
