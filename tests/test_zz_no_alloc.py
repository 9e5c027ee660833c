"""festung_apply_noalloc: the apply variant for callers that cannot allocate device
memory (an external pool owns the device memory, or cudaMalloc's implicit
synchronisation is not allowed).  Called through the C ABI and compared with
festung_apply on two calls in a row; collected last so that a stop-at-first-failure
run has already run every other test."""
import ctypes

import numpy as np
import pytest

from helpers import gpu_solver, mesh, samples, smooth_d

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _call(s, fn, x, y, prec, dt):
    rc = fn(s.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), prec, ctypes.c_double(dt))
    return rc


@pytest.mark.parametrize("p", [1, 3])
def test_noalloc_matches_apply_twice(p):
    import torch
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(20, "mixed", seed=3)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_coeff(samples(s, smooth_d))
    lib = s.lib
    for prec, dtype, eps in ((F.FP64, torch.float64, EPS64), (F.FP32, torch.float32, EPS32)):
        for call in range(2):
            x = torch.randn(s.N, s.K, dtype=dtype, device="cuda", generator=torch.Generator("cuda").manual_seed(call))
            y_ref = torch.empty_like(x)
            y_na = torch.full_like(x, float("nan"))
            assert _call(s, lib.festung_apply, x, y_ref, prec, 0.02) == F.OK
            assert _call(s, lib.festung_apply_noalloc, x, y_na, prec, 0.02) == F.OK, \
                lib.festung_last_error(s.h).decode()
            torch.cuda.synchronize()
            scale = y_ref.abs().max().item()
            assert torch.isfinite(y_na).all()
            assert (y_na - y_ref).abs().max().item() <= 64 * eps * scale
    s.close()


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch():
    import torch
    from paper_1408_3877_gb300 import festung as F
    # 2 x N x K x 8 B = 2 x 15 x 140,450 x 8 B = 33.7 MB > 32 MiB in FP64; 16.9 MB fits in FP32
    cV, V0T, bdr = mesh(265, "neumann", seed=1)
    s = gpu_solver(cV, V0T, bdr, 4)
    x = torch.zeros(s.N, s.K, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    assert _call(s, s.lib.festung_apply_noalloc, x, y, F.FP64, 0.01) == F.EINVAL
    assert "32" in s.lib.festung_last_error(s.h).decode() or "bytes" in s.lib.festung_last_error(s.h).decode()
    # the FP32 case near the limit, on seeded random data against festung_apply
    g = torch.Generator("cuda").manual_seed(5)
    xf = torch.randn(s.N, s.K, dtype=torch.float32, device="cuda", generator=g)
    yf = torch.full_like(xf, float("nan"))
    yr = torch.empty_like(xf)
    assert _call(s, s.lib.festung_apply_noalloc, xf, yf, F.FP32, 0.01) == F.OK
    assert _call(s, s.lib.festung_apply, xf, yr, F.FP32, 0.01) == F.OK
    torch.cuda.synchronize()
    assert torch.isfinite(yf).all()
    assert (yf - yr).abs().max().item() <= 64 * EPS32 * yr.abs().max().item()
    s.close()


def test_noalloc_first_call_on_a_fresh_context_allocates_nothing():
    """The entry point as the very first apply of a new context (nothing has allocated the
    context's apply workspace yet), then a second call: both match festung_apply, and the
    second call leaves the device's free memory unchanged."""
    import torch
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(24, "dirichlet", seed=9)
    s = gpu_solver(cV, V0T, bdr, 2)
    s.set_coeff(samples(s, smooth_d))
    g = torch.Generator("cuda").manual_seed(11)
    x = torch.randn(s.N, s.K, dtype=torch.float64, device="cuda", generator=g)
    y1, y2, yr = (torch.full_like(x, float("nan")) for _ in range(3))
    assert _call(s, s.lib.festung_apply_noalloc, x, y1, F.FP64, 0.005) == F.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _call(s, s.lib.festung_apply_noalloc, x, y2, F.FP64, 0.005) == F.OK
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert _call(s, s.lib.festung_apply, x, yr, F.FP64, 0.005) == F.OK
    torch.cuda.synchronize()
    scale = yr.abs().max().item()
    for y in (y1, y2):
        assert torch.isfinite(y).all()
        assert (y - yr).abs().max().item() <= 64 * EPS64 * scale
    s.close()
