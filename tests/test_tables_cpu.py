"""Host logic of the CUDA library: its quadrature rules and basis tables (tables.cpp),
compiled natively here and checked against exact moments and orthonormality.  These
pins do not use the oracle."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1408_3877_gb300", "csrc")


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("tab") / "tables_check")
    inc = ["-I" + CSRC, "-I" + os.path.join(ROOT, "include"), "-I/usr/local/cuda/include"]
    subprocess.run([cxx, "-std=c++17", "-O2", *inc, os.path.join(ROOT, "tests", "native", "tables_check.cpp"),
                    os.path.join(CSRC, "tables.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return [line.split() for line in out.splitlines()]


def test_triangle_rules_exact(report):
    rows = [r for r in report if r[0] == "tri"]
    assert len(rows) == 10
    for _, q, npts, worst, minw, minx in rows:
        assert float(worst) < 1e-14, (q, worst)
        assert float(minw) > 0 and float(minx) > 0, q
    sizes = {int(r[1]): int(r[2]) for r in rows}
    assert sizes[1] == 1 and sizes[2] == 3 and sizes[4] == 6 and sizes[5] == 7 and sizes[6] == 12
    assert sizes[8] == 25 and sizes[7] == 16


def test_gauss_rules_exact_and_symmetric(report):
    for _, n, worst, sym in [r for r in report if r[0] == "gauss"]:
        assert float(worst) < 1e-14, n
        assert float(sym) == 0.0, n


def test_basis_orthonormal_and_signs(report):
    row = [r for r in report if r[0] == "basis"][0]
    assert float(row[1]) < 1e-12 and float(row[2]) < 1e-6
    # sign of phi_i(0, 0) in the paper's basis (Sec. 2.4.1 closed forms and routine phi)
    assert [int(v) for v in row[3:]] == [1, 1, 1, 1, -1, 1, -1, -1, -1, -1, 1, 1, 1, 1, 1]
