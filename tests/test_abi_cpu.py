"""CPU checks of the C ABI: the library loads, exports every declared symbol, and
rejects invalid meshes before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "festung.h")).read()
    return sorted(set(re.findall(r"\b(festung_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1408_3877_gb300 import festung as F
    if not os.path.exists(F.LIB_PATH):
        from paper_1408_3877_gb300 import build
        build.build()
    return F.load()


def test_exports_every_declared_symbol(lib):
    from paper_1408_3877_gb300 import festung as F
    names = _declared()
    assert set(names) == set(F.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_constants_match_the_header():
    from paper_1408_3877_gb300 import festung as F
    txt = open(os.path.join(ROOT, "include", "festung.h")).read()
    defs = dict(re.findall(r"#define\s+FESTUNG_([A-Z0-9_]+)\s+(-?\d+)\b", txt))
    assert len(defs) >= 20
    for name, value in defs.items():
        assert getattr(F, name) == int(value), name


def _create(lib, cV, V0T, bdr):
    cV = np.ascontiguousarray(cV, dtype=np.float64)
    V0T = np.ascontiguousarray(V0T, dtype=np.int32)
    bdr = np.ascontiguousarray(bdr, dtype=np.int8)
    h = ctypes.c_void_p()
    rc = lib.festung_mesh_create(cV.ctypes.data, cV.shape[0], V0T.ctypes.data, V0T.shape[0], bdr.ctypes.data,
                                 ctypes.byref(h))
    return rc, lib.festung_last_error(None).decode()


def test_invalid_meshes_rejected_on_host(lib):
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, side = W.square_mesh(3)
    bdr = W.boundary_types(side, (1, 2, 3, 4))
    rc, msg = _create(lib, cV, V0T[:, ::-1], bdr)
    assert rc == F.EMESH and "clockwise" in msg
    bad = bdr.copy()
    bad[bad > 0] = 0
    rc, msg = _create(lib, cV, V0T, bad)
    assert rc == F.EMESH and "boundary" in msg
    bad = bdr.copy()
    k, n = np.argwhere(bdr == 0)[0]
    bad[k, n] = 1
    rc, msg = _create(lib, cV, V0T, bad)
    assert rc == F.EMESH and "interior" in msg
    cV2 = cV.copy()
    cV2[0, 0] = np.nan
    rc, _ = _create(lib, cV2, V0T, bdr)
    assert rc == F.EDATA
    V2 = V0T.copy()
    V2[0, 0] = 10**6
    rc, _ = _create(lib, cV, V2, bdr)
    assert rc == F.EMESH
    # an edge used by three triangles
    V3 = np.concatenate([V0T, V0T[:1, [1, 0, 2]]])
    b3 = np.concatenate([bdr, bdr[:1]])
    rc, _ = _create(lib, cV, V3, b3)
    assert rc == F.EMESH


def test_null_arguments(lib):
    from paper_1408_3877_gb300 import festung as F
    h = ctypes.c_void_p()
    assert lib.festung_mesh_create(None, 0, None, 0, None, ctypes.byref(h)) == F.EINVAL
    assert lib.festung_setup(None, 1, 0, 1.0) == F.EINVAL
    lib.festung_destroy(None)


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: the header compiles as strict C99 (no C++ or CUDA types)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "festung.h"\nint main(void) { festung_ctx *c = 0; (void)c; return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        "-fsyntax-only", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
