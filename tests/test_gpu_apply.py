"""Parity of the CUDA operator apply y = S x (E1) with the oracle's CSR product.

FP64: |y_gpu - y_oracle| is bounded by a small multiple of the rounding scale
eps64 |S| |x| in 2-norm, and element by element by a small multiple of eps64 times the
factored scale |M| |x| + tau (eta |S_t| |x| + sum_m |A_m| |M^{-1}| |B_m| |x|) (the two
sides sum the same quadrature terms in different orders and groupings; the kernels
evaluate S in factors, the flux unknowns first).
FP32: the same bound with eps32 (geometry, tables, D and x rounded to FP32).
Double-float (FESTUNG_DFLOAT): the same bound with 2^-47 (value = hi + lo of two
FP32 numbers; inputs split with 2^-48 relative error, sums and products with errors
of a few units of 2^-48 of the operand magnitudes).
"""
import numpy as np
import pytest

from helpers import (factored_scale, from_gpu_layout, gpu_solver, mesh, patch_oracle_rows, rounding_bound, samples,
                     smooth_d, to_gpu_layout)

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps
EPSDF = 2.0 ** -47


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _case(n, p, mix, tau, quad_order=None, seed=1, jitter=0.2):
    import torch
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(n, mix, jitter=jitter, seed=seed)
    L = LDG(cV, V0T, bdr, p, quad_order=quad_order)
    s = gpu_solver(cV, V0T, bdr, p, quad_order or 0)
    s.set_coeff(samples(s, smooth_d))
    D = L.project(smooth_d)
    S = L.operator(D, tau)
    x = np.random.default_rng(seed + 7).standard_normal(L.K * L.N)
    y_or = S @ x
    out = {}
    order = s.element_order()
    for prec, dt in ((F.FP64, torch.float64), (F.FP32, torch.float32), (F.DFLOAT, torch.float64)):
        xg = to_gpu_layout(x, L.K, L.N, dt, order)
        yg = torch.empty_like(xg)
        s.apply(xg, yg, tau, prec)
        torch.cuda.synchronize()
        out[prec] = from_gpu_layout(yg, order).ravel()
    s.close()
    return S, x, y_or, out, factored_scale(L, D, tau, x)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mix", ["dirichlet", "neumann", "mixed"])
def test_apply_matches_oracle(p, mix):
    from paper_1408_3877_gb300 import festung as F
    # n = 13: K = 338 spans two 256-thread blocks with a ragged tail
    S, x, y, out, scale = _case(13, p, mix, tau=0.01)
    bound = rounding_bound(abs(S), x, 1.0)
    e64 = np.linalg.norm(out[F.FP64] - y)
    e32 = np.linalg.norm(out[F.FP32] - y)
    assert e64 <= 64 * EPS64 * bound, (e64, bound)
    assert e32 <= 64 * EPS32 * bound, (e32, bound)
    # element by element
    assert np.all(np.abs(out[F.FP64] - y) <= 256 * EPS64 * (scale + 1e-300)), \
        np.max(np.abs(out[F.FP64] - y) / (scale + 1e-300))
    assert np.all(np.abs(out[F.DFLOAT] - y) <= 256 * EPSDF * (scale + 1e-300)), \
        np.max(np.abs(out[F.DFLOAT] - y) / (scale + 1e-300))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_apply_quadrature_2p_plus_1(p):
    from paper_1408_3877_gb300 import festung as F
    S, x, y, out, _ = _case(6, p, "mixed", tau=0.05, quad_order=2 * p + 1)
    bound = rounding_bound(abs(S), x, 1.0)
    assert np.linalg.norm(out[F.FP64] - y) <= 64 * EPS64 * bound


def test_apply_dt_zero_is_mass_and_two_triangles():
    import torch
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    r3 = np.sqrt(3.0)
    cV = np.array([[0.0, -1.0], [r3, 0.0], [0.0, 1.0], [-r3, 0.0]])
    V0T = np.array([[3, 0, 2], [0, 1, 2]])
    bdr = np.array([[0, 1, 2], [2, 0, 1]])
    for p in range(5):
        L = LDG(cV, V0T, bdr, p)
        s = gpu_solver(cV, V0T, bdr, p)
        s.set_coeff(samples(s, smooth_d))
        x = np.random.default_rng(p).standard_normal(2 * L.N)
        for tau in (0.0, 0.3):
            y = L.operator(L.project(smooth_d), tau) @ x
            order = s.element_order()
            xg = to_gpu_layout(x, 2, L.N, torch.float64, order)
            yg = torch.empty_like(xg)
            s.apply(xg, yg, tau, F.FP64)
            torch.cuda.synchronize()
            assert np.allclose(from_gpu_layout(yg, order).ravel(), y, rtol=1e-12, atol=1e-12 * np.abs(y).max())
        s.close()


def test_apply_deterministic_bitwise():
    import torch
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(24, "mixed")
    s = gpu_solver(cV, V0T, bdr, 3)
    s.set_coeff(samples(s, smooth_d))
    x = torch.randn(s.N, s.K, dtype=torch.float64, device="cuda")
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    s.apply(x, y1, 0.01, F.FP64)
    s.apply(x, y2, 0.01, F.FP64)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    s.close()


@pytest.mark.parametrize("cfg", ["grf1024_p2", "jitter256_p4"])
def test_apply_full_size_sampled(cfg):
    """Full-size workloads, launched as the bench launches them: sampled rows against the
    oracle evaluated on the 2-ring patch of each sampled triangle, plus conservation and
    the constant state on the all-Neumann workload."""
    import torch
    import workloads as W
    from paper_1408_3877_gb300 import festung as F
    c = W.CONFIGS[cfg]
    cV, V0T, side = W.square_mesh(c["n"], jitter=c["jitter"], seed=11)
    bdr = W.boundary_types(side, c["dirichlet"], c["neumann"])
    p, tau = c["p"], c["dt"]
    if c["coeff"] == "grf":
        g = W.GaussianField(5, c["grf_length"])
        dfun = lambda x, y: np.exp(g(x, y))
    else:
        dfun = lambda x, y: W.d_config2(0.5, x, y)[0]
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_coeff(samples(s, dfun))
    K, N = s.K, s.N
    rng = np.random.default_rng(3)
    x = rng.standard_normal((K, N))
    ks = rng.choice(K, 24, replace=False)
    rows, scale = patch_oracle_rows(cV, V0T, bdr, p, dfun, x, tau, ks)
    order = s.element_order()
    for prec, dt, eps in ((F.FP64, torch.float64, EPS64), (F.FP32, torch.float32, EPS32)):
        xg = to_gpu_layout(x, K, N, dt, order)
        yg = torch.empty_like(xg)
        s.apply(xg, yg, tau, prec)
        torch.cuda.synchronize()
        y = from_gpu_layout(yg, order)
        err = np.abs(y[ks] - rows)
        assert np.all(err <= 256 * eps * scale), (prec, (err / scale).max())
    if not c["dirichlet"]:
        xs = to_gpu_layout(x, K, N, torch.float64, order)
        y0, y1 = torch.empty_like(xs), torch.empty_like(xs)
        s.apply(xs, y0, 0.0, F.FP64)
        s.apply(xs, y1, tau, F.FP64)
        torch.cuda.synchronize()
        tot = (y1 - y0)[0].sum().item()
        assert abs(tot) <= 1e-9 * (y1 - y0).abs().max().item() * np.sqrt(K)
        one = torch.zeros_like(xs)
        one[0] = 1.0
        s.apply(one, y0, 0.0, F.FP64)
        s.apply(one, y1, tau, F.FP64)
        torch.cuda.synchronize()
        assert (y1 - y0).abs().max().item() <= 1e-9 * y0.abs().max().item()
    s.close()


def test_autotune_changes_only_the_tiling():
    import torch
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(40, "mixed", seed=6)   # 3200 triangles: several tiles at every candidate size
    s = gpu_solver(cV, V0T, bdr, 3)
    s.set_coeff(samples(s, smooth_d))
    x = torch.randn(s.N, s.K, dtype=torch.float64, device="cuda")
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    s.apply(x, y0, 0.01, F.FP64)
    te = s.autotune()
    assert te in range(96, 257, 32)
    s.apply(x, y1, 0.01, F.FP64)
    torch.cuda.synchronize()
    assert float((y1 - y0).abs().max()) <= 1e-12 * float(y0.abs().max())
    s.close()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_apply_bf16_tables_within_their_rounding(p):
    """FESTUNG_BF16TAB: every reference table entry rounded to BF16 (relative error <= 2^-9),
    FP32 data and sums.  Each term of the factored evaluation is a product of at most three
    table entries, so the result stays within 4 * 2^-9 of the factored scale; and it must
    differ from the FP32 operator (the tables really are the rounded ones).  At p >= 3 the
    volume term runs on the tensor cores (TF32-split operands, about 2^-20 relative)."""
    import torch
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(13, "mixed", seed=1)
    L = LDG(cV, V0T, bdr, p)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_coeff(samples(s, smooth_d))
    D = L.project(smooth_d)
    tau = 0.01
    y = L.operator(D, tau) @ (x := np.random.default_rng(3).standard_normal(L.K * L.N))
    scale = factored_scale(L, D, tau, x)
    order = s.element_order()
    xg = to_gpu_layout(x, L.K, L.N, torch.float32, order)
    out = {}
    for prec in (F.FP32, F.BF16TAB):
        yg = torch.empty_like(xg)
        s.apply(xg, yg, tau, prec)
        torch.cuda.synchronize()
        out[prec] = from_gpu_layout(yg, order).ravel()
    s.close()
    err = np.abs(out[F.BF16TAB] - y)
    assert np.all(err <= 4 * 2.0 ** -9 * scale + 64 * EPS32 * scale), np.max(err / scale)
    assert np.max(np.abs(out[F.BF16TAB] - out[F.FP32]) / scale) > 1e-5
