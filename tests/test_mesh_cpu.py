"""Host logic of the CUDA library: mesh validation, the Morton renumbering and the
tiles with their halos (mesh.cpp), compiled natively and checked for consistency."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1408_3877_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("mesh") / "mesh_check")
    inc = ["-I" + CSRC, "-I" + os.path.join(ROOT, "include"), "-I/usr/local/cuda/include"]
    subprocess.run([cxx, "-std=c++17", "-O2", *inc, os.path.join(ROOT, "tests", "native", "mesh_check.cpp"),
                    os.path.join(CSRC, "mesh.cpp"), "-o", out], check=True)
    return out


@pytest.mark.parametrize("n,te", [(13, 64), (24, 256), (40, 256), (7, 1000)])
def test_order_and_tiles(exe, n, te):
    r = subprocess.run([exe, str(n), str(te)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok perm" in r.stdout and "ok neighbours" in r.stdout and "ok tiles" in r.stdout and "ok lift" in r.stdout
    assert "ok tile_size" in r.stdout
