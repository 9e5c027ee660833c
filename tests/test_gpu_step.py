"""Parity of the CUDA implicit-Euler step with the oracle's sparse direct solve of the
3KN system (Sec. 2.5).  FP64 path at Krylov tolerance 1e-13: relative L2 difference
<= 1e-11 per step.  Mixed path (FP32 inner solve, refinement on double-float residuals) at tolerance 1e-12:
<= 1e-9.  The solution error of an iterative solve is at most cond(S) * tol; the
meshes here have cond(S) <= ~1e2 after the mass scaling."""
import numpy as np
import pytest

import workloads as W
from helpers import edge_samples, gpu_solver, mesh, samples, smooth_d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _load_step_data(s, man, t):
    s.set_coeff(samples(s, lambda x, y: man.d(t, x, y)))
    s.set_source(samples(s, lambda x, y: man.f(t, x, y)))
    s.set_bc(edge_samples(s, lambda x, y: man.c(t, x, y)), edge_samples(s, lambda x, y: man.gN(t, x, y)))


def _oracle_step(L, man, C, t, tau):
    return L.step(C, L.project(lambda x, y: man.d(t, x, y)), L.project(lambda x, y: man.f(t, x, y)),
                  lambda x, y: man.c(t, x, y), lambda x, y: man.gN(t, x, y), tau)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mix", ["dirichlet", "neumann", "mixed"])
def test_step_fp64_matches_oracle(p, mix):
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(6, mix, seed=2)
    man = W.Manufactured(W.d_config2)
    tau, t = 0.01, 0.01
    L = LDG(cV, V0T, bdr, p)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    _load_step_data(s, man, t)
    info = s.step(tau, tol=1e-13, prec=F.FP64)
    C = s.get_state()
    Co = _oracle_step(L, man, L.project(lambda x, y: man.c(0.0, x, y)), t, tau)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-11, (err, info)
    assert info["rel_residual"] <= 1e-13
    if p == 0:  # d_h is elementwise constant for p = 0: S is symmetric, CG
        assert info["solver"] == F.SOLVER_CG and info["symmetric"] == 1
    else:
        assert info["solver"] == F.SOLVER_BICGSTAB and info["symmetric"] == 0
    s.close()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_step_mixed_matches_oracle(p):
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(10, "mixed", seed=4)
    man = W.Manufactured(W.d_config2)
    tau, t = 0.005, 0.005
    L = LDG(cV, V0T, bdr, p)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    _load_step_data(s, man, t)
    info = s.step(tau, tol=1e-12, prec=F.MIXED, inner_tol=1e-3)
    C = s.get_state()
    Co = _oracle_step(L, man, L.project(lambda x, y: man.c(0.0, x, y)), t, tau)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-9, (err, info)
    assert info["outer"] >= 2
    assert info["fp64_iterations"] == 0, info  # the FP32 sweeps converge without the FP64 fallback
    s.close()


@pytest.mark.parametrize("p", [1, 4])
def test_mixed_residual_holds_in_fp64(p):
    """The mixed step certifies its tolerance with residuals evaluated in double-float
    arithmetic; its result must meet the same tolerance in FP64.  With C_ref from an
    FP64 solve at 1e-14, b - S C = S (C_ref - C) + r_ref, and S (C_ref - C) is applied
    in FP64 to the (small) difference."""
    import torch
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, side = W.square_mesh(24, jitter=0.2, seed=8)
    bdr = W.boundary_types(side, (2, 4), (1, 3))
    man = W.Manufactured(W.d_config2)
    tau, t = 1e-3, 1e-3
    res = {}
    for prec, tol in ((F.FP64, 1e-14), (F.MIXED, 1e-10)):
        s = gpu_solver(cV, V0T, bdr, p)
        s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
        _load_step_data(s, man, t)
        info = s.step(tau, tol=tol, prec=prec, inner_tol=1e-2)
        res[prec] = (s.get_state(), info)
        if prec == F.FP64:
            order = s.element_order()
            keep = s
        else:
            s.close()
    from helpers import from_gpu_layout, to_gpu_layout
    Cref, Cmix = res[F.FP64][0], res[F.MIXED][0]
    K, N = keep.K, keep.N
    x = to_gpu_layout(Cref.ravel(), K, N, torch.float64, order)
    b = torch.empty_like(x)
    keep.apply(x, b, tau, F.FP64)                      # S C_ref = b up to 1e-14 ||b||
    dx = to_gpu_layout((Cref - Cmix).ravel(), K, N, torch.float64, order)
    r = torch.empty_like(dx)
    keep.apply(dx, r, tau, F.FP64)
    torch.cuda.synchronize()
    rel = float(torch.linalg.norm(r) / torch.linalg.norm(b))
    assert res[F.FP64][1]["rel_residual"] <= 1e-14
    assert rel <= 1.2e-10, (rel, res[F.MIXED][1])
    keep.close()


@pytest.mark.parametrize("p", [2, 4])
def test_mixed_sweeps_converge_like_fp64(p):
    """The FP32 BiCGStab sweeps (reductions fused into the applies) need about as many
    iterations as the FP64 BiCGStab for the same reduction, and no FP64 fallback."""
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, side = W.square_mesh(32, jitter=0.2, seed=6)
    bdr = W.boundary_types(side, (2, 4), (1, 3))
    man = W.Manufactured(W.d_config2)
    tau, t = 1e-3, 1e-3
    its = {}
    for prec in (F.FP64, F.MIXED):
        s = gpu_solver(cV, V0T, bdr, p)
        s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
        _load_step_data(s, man, t)
        info = s.step(tau, tol=1e-10, prec=prec, inner_tol=1e-2)
        assert info["rel_residual"] <= 1e-10
        its[prec] = info
        s.close()
    assert its[F.MIXED]["fp64_iterations"] == 0, its
    assert its[F.MIXED]["iterations"] <= 2 * its[F.FP64]["iterations"] + 10, its


def test_square8_p1_ten_steps():
    """The 8x8 workload: p = 1, triangle rule of degree 3 (served by the degree-4 rule),
    Dirichlet data from c on the whole boundary, dt = 0.01 for 10 steps; every step is
    compared with the oracle's solve of eq. fullSystem."""
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    c = W.CONFIGS["square8_p1"]
    cV, V0T, side = W.square_mesh(c["n"])
    bdr = W.boundary_types(side, c["dirichlet"], c["neumann"])
    man = W.Manufactured(W.d_config1)
    L = LDG(cV, V0T, bdr, c["p"], quad_order=c["quad_order"])
    s = gpu_solver(cV, V0T, bdr, c["p"], c["quad_order"])
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    Co = L.project(lambda x, y: man.c(0.0, x, y))
    for n in range(1, c["steps"] + 1):
        t = n * c["dt"]
        _load_step_data(s, man, t)
        s.step(c["dt"], tol=1e-13, prec=F.FP64)
        D = L.project(lambda x, y: man.d(t, x, y))
        Fh = L.project(lambda x, y: man.f(t, x, y))
        Co, _, _ = L.step_full(Co, D, Fh, lambda x, y: man.c(t, x, y), None, c["dt"])
        C = s.get_state()
        assert np.linalg.norm(C - Co) <= 1e-11 * np.linalg.norm(Co), n
    # the discrete solution tracks the exact one
    err = s.l2_error(samples(s, lambda x, y: man.c(c["steps"] * c["dt"], x, y)))
    assert err < 5e-2
    s.close()


def test_symmetric_case_uses_cg():
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(8, "mixed", seed=5)
    p, tau = 2, 0.02
    s = gpu_solver(cV, V0T, bdr, p)
    rng = np.random.default_rng(9)
    dk = rng.uniform(0.5, 2.0, s.K)
    s.set_coeff(np.repeat(dk[:, None], s.R2, axis=1))        # d elementwise constant
    s.set_state(samples(s, lambda x, y: np.sin(3 * x) * y), is_samples=True)
    s.set_bc(edge_samples(s, lambda x, y: x + y), edge_samples(s, lambda x, y: 0 * x + 0.5))
    info = s.step(tau, tol=1e-13, prec=F.FP64)
    assert info["symmetric"] == 1 and info["solver"] == F.SOLVER_CG
    L = LDG(cV, V0T, bdr, p)
    D = L.project(lambda x, y: 0 * x + 1.0) * dk[:, None]
    C0 = L.project(lambda x, y: np.sin(3 * x) * y)
    Co = L.step(C0, D, None, lambda x, y: x + y, lambda x, y: 0 * x + 0.5, tau)
    C = s.get_state()
    assert np.linalg.norm(C - Co) <= 1e-11 * np.linalg.norm(Co)
    s.close()


def test_errors_leave_state_unchanged():
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(6, "mixed")
    s = gpu_solver(cV, V0T, bdr, 2)
    s.set_state(samples(s, lambda x, y: np.cos(x) * y), is_samples=True)
    C0 = s.get_state()
    d = samples(s, smooth_d)
    s.set_coeff(d)
    bad = d.copy()
    bad[3, 1] = -1.0
    with pytest.raises(F.FestungError) as e:
        s.set_coeff(bad)
    assert e.value.code == F.EDATA
    bad[3, 1] = np.nan
    with pytest.raises(F.FestungError) as e:
        s.set_coeff(bad)
    assert e.value.code == F.EDATA
    with pytest.raises(F.FestungError) as e:
        s.step(0.01, tol=1e-14, prec=F.FP64, max_iter=1, max_outer=1)
    assert e.value.code == F.ENOCONV
    assert np.array_equal(s.get_state(), C0)
    with pytest.raises(F.FestungError) as e:
        s.step(-1.0)
    assert e.value.code == F.EINVAL
    s.close()


@pytest.mark.parametrize("p", [0, 2, 4])
def test_single_triangle_step(p):
    """The smallest mesh: one triangle, Dirichlet on two edges and Neumann on one (no
    interior edge, one tile of one triangle, no halo)."""
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
    V0T = np.array([[0, 1, 2]])
    bdr = np.array([[1, 2, 1]])
    man = W.Manufactured(W.d_config2)
    tau, t = 0.01, 0.01
    L = LDG(cV, V0T, bdr, p)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    _load_step_data(s, man, t)
    for prec, tol, bound in ((F.FP64, 1e-13, 1e-11), (F.MIXED, 1e-12, 1e-9)):
        s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
        info = s.step(tau, tol=tol, prec=prec)
        C = s.get_state()
        Co = _oracle_step(L, man, L.project(lambda x, y: man.c(0.0, x, y)), t, tau)
        assert np.linalg.norm(C - Co) <= bound * np.linalg.norm(Co), (prec, info)
    s.close()


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("prec_name,tol,bound", [("FP64", 1e-13, 1e-10), ("MIXED", 1e-12, 1e-9)])
def test_step_reproduces_discrete_solutions_linear_in_time(p, prec_name, tol, bound):
    """The step's patch test (Sec. 2.5, consistency of LDG and of the implicit-Euler
    quotient for c linear in t) on the GPU, against the GPU's own projection of c(t_n+1):
    no oracle value enters."""
    from helpers import patch_case
    from paper_1408_3877_gb300 import festung as F
    c0, d, f0, gN0 = patch_case(p)
    c1, _, f1, gN1 = patch_case(1)
    cV, V0T, side = W.square_mesh(8, jitter=0.2, seed=5)
    bdr = W.boundary_types(side, (2, 4), (1, 3))
    s = gpu_solver(cV, V0T, bdr, p)
    tn, tau = 0.3, 0.05
    t = tn + tau
    s.set_state(samples(s, lambda x, y: c0(x, y) + t * c1(x, y)), is_samples=True)
    Cp = s.get_state()
    s.set_state(samples(s, lambda x, y: c0(x, y) + tn * c1(x, y)), is_samples=True)
    s.set_coeff(samples(s, d))
    s.set_source(samples(s, lambda x, y: c1(x, y) + f0(x, y) + t * f1(x, y)))
    s.set_bc(edge_samples(s, lambda x, y: c0(x, y) + t * c1(x, y)),
             edge_samples(s, lambda x, y: gN0(x, y) + t * gN1(x, y)))
    info = s.step(tau, tol=tol, prec=getattr(F, prec_name), inner_tol=1e-3)
    C = s.get_state()
    err = np.linalg.norm(C - Cp) / np.linalg.norm(Cp)
    assert err <= bound, (err, info)
    s.close()
