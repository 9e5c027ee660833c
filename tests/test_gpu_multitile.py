"""Step parity with the oracle on meshes that the library splits into several tiles.

A 32 x 32 jittered grid has 2,048 triangles.  The fused apply takes tiles of at most 256
triangles, so every apply runs 8 tiles with halos: the neighbour traces across tile
borders come from the halo slots (and, for a halo triangle's own outer neighbours, from
global memory), and every Krylov reduction sums the partials of several blocks before
the last block updates the scalars.  The small meshes of the other step tests run as
one tile and do not reach these paths.

Each step is compared element by element with the oracle's sparse direct solve of the
eliminated system (Sec. 2.5, eq. fullSystem with z eliminated), on the same seeded
inputs: FP64 at Krylov tolerance 1e-13 within 1e-11 relative L2; the mixed path (FP32
inner iterations, refinement on double-float residuals) at 1e-12 within 1e-9, for
p = 0..4 including the p = 4 order of the benchmark."""
import numpy as np
import pytest

import workloads as W
from helpers import edge_samples, gpu_solver, mesh, samples

pytestmark = pytest.mark.gpu

MESH_N = 32
TAU = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


_ORACLE = {}


def _oracle(p, mix, man, t):
    """C^1 of the oracle from the projection of c(0) (cached per order and boundary mix)."""
    key = (p, mix)
    if key not in _ORACLE:
        from oracle.solve import LDG
        cV, V0T, bdr = mesh(MESH_N, mix, seed=21)
        L = LDG(cV, V0T, bdr, p)
        C0 = L.project(lambda x, y: man.c(0.0, x, y))
        _ORACLE[key] = L.step(C0, L.project(lambda x, y: man.d(t, x, y)), L.project(lambda x, y: man.f(t, x, y)),
                              lambda x, y: man.c(t, x, y), lambda x, y: man.gN(t, x, y), TAU)
    return _ORACLE[key]


def _gpu_step(p, mix, man, t, prec, tol, coarse=False, **kw):
    cV, V0T, bdr = mesh(MESH_N, mix, seed=21)
    s = gpu_solver(cV, V0T, bdr, p)
    if coarse:
        s.set_coarse(True)
    assert s.K == 2 * MESH_N ** 2
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    s.set_coeff(samples(s, lambda x, y: man.d(t, x, y)))
    s.set_source(samples(s, lambda x, y: man.f(t, x, y)))
    s.set_bc(edge_samples(s, lambda x, y: man.c(t, x, y)), edge_samples(s, lambda x, y: man.gN(t, x, y)))
    info = s.step(TAU, tol=tol, prec=prec, **kw)
    C = s.get_state()
    s.close()
    return C, info


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_multitile_fp64_step_matches_oracle(p):
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    C, info = _gpu_step(p, "mixed", man, TAU, F.FP64, 1e-13)
    Co = _oracle(p, "mixed", man, TAU)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-11, (err, info)
    assert info["rel_residual"] <= 1e-13


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_multitile_mixed_step_matches_oracle(p):
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    C, info = _gpu_step(p, "mixed", man, TAU, F.MIXED, 1e-12, inner_tol=1e-2)
    Co = _oracle(p, "mixed", man, TAU)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-9, (err, info)
    assert info["rel_residual"] <= 1e-12
    assert info["fp64_iterations"] == 0, info  # the FP32 sweeps alone reach the tolerance


@pytest.mark.parametrize("mix", ["dirichlet", "neumann"])
def test_multitile_boundary_mixes_match_oracle(mix):
    """All-Dirichlet and all-Neumann boundaries across tile borders, p = 2, both precisions."""
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    Co = _oracle(2, mix, man, TAU)
    for prec, tol, bound in ((F.FP64, 1e-13, 1e-11), (F.MIXED, 1e-12, 1e-9)):
        C, info = _gpu_step(2, mix, man, TAU, prec, tol)
        err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
        assert err <= bound, (prec, err, info)


def test_multitile_stationary_matches_oracle():
    """The stationary problem of Sec. 3.9 (no mass term) on the multi-tile mesh, p = 3."""
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(MESH_N, "mixed", seed=21)
    man = W.Manufactured(W.d_verification, stationary=True)
    p = 3
    L = LDG(cV, V0T, bdr, p)
    Co = L.stationary(L.project(lambda x, y: man.d(0.0, x, y)), L.project(lambda x, y: man.f(0.0, x, y)),
                      lambda x, y: man.c(0.0, x, y), lambda x, y: man.gN(0.0, x, y))
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_coeff(samples(s, lambda x, y: man.d(0.0, x, y)))
    s.set_source(samples(s, lambda x, y: man.f(0.0, x, y)))
    s.set_bc(edge_samples(s, lambda x, y: man.c(0.0, x, y)), edge_samples(s, lambda x, y: man.gN(0.0, x, y)))
    info = s.solve_stationary(tol=1e-13, prec=F.FP64)
    err = np.linalg.norm(s.get_state() - Co) / np.linalg.norm(Co)
    s.close()
    # without the mass term cond(S) grows like h^-2 (~1e4-1e5 here): error <= cond(S) tol
    assert err <= 1e-8, (err, info)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_multitile_mixed64_step_matches_oracle(p):
    """FESTUNG_MIXED64: FP32 inner sweeps with the refinement residual in FP64."""
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    C, info = _gpu_step(p, "mixed", man, TAU, F.MIXED64, 1e-12, inner_tol=1e-2)
    Co = _oracle(p, "mixed", man, TAU)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-9, (err, info)
    assert info["rel_residual"] <= 1e-12
    assert info["outer"] >= 2 and info["fp64_iterations"] == 0, info


@pytest.mark.parametrize("p", [1, 2])
def test_multitile_bf16_table_step_matches_oracle(p):
    """FESTUNG_BF16TAB: inner sweeps on the operator with BF16-rounded tables; the FP64
    refinement still reaches the tolerance on the exact operator, so the result matches
    the oracle like the other modes (at the cost of more sweeps)."""
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    C, info = _gpu_step(p, "mixed", man, TAU, F.BF16TAB, 1e-12, inner_tol=1e-2)
    Cm, info_m = _gpu_step(p, "mixed", man, TAU, F.MIXED, 1e-12, inner_tol=1e-2)
    Co = _oracle(p, "mixed", man, TAU)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-9, (err, info)
    assert info["rel_residual"] <= 1e-12
    assert info["outer"] >= info_m["outer"], (info, info_m)  # BF16 tables need at least as many sweeps


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("prec_name", ["MIXED", "MIXED64"])
def test_multitile_coarse_corrected_step_matches_oracle(p, prec_name):
    """festung_set_coarse: every FP32 sweep starts from the p = 1 coarse correction; the step
    still matches the oracle within the mixed bound (the answer does not depend on it)."""
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    C, info = _gpu_step(p, "mixed", man, TAU, getattr(F, prec_name), 1e-12, coarse=True, inner_tol=1e-2)
    Co = _oracle(p, "mixed", man, TAU)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-9, (err, info)
    assert info["rel_residual"] <= 1e-12
    assert info["coarse_iterations"] > 0 and info["fp64_iterations"] == 0, info


@pytest.mark.parametrize("p", [0, 1])
def test_multitile_persistent_and_graph_iterations_match_oracle(p):
    """festung_set_persistent: at p <= 1 the FP32 BiCGStab iterations run as one persistent
    kernel (default) or as the graph of four kernels per iteration; on the 8-tile mesh both
    reach the oracle's step within the mixed bound, with about the same iteration count
    (their sums round differently)."""
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    Co = _oracle(p, "mixed", man, TAU)
    out = {}
    for persistent in (True, False):
        cV, V0T, bdr = mesh(MESH_N, "mixed", seed=21)
        s = gpu_solver(cV, V0T, bdr, p)
        s.set_persistent(persistent)
        s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
        s.set_coeff(samples(s, lambda x, y: man.d(TAU, x, y)))
        s.set_source(samples(s, lambda x, y: man.f(TAU, x, y)))
        s.set_bc(edge_samples(s, lambda x, y: man.c(TAU, x, y)), edge_samples(s, lambda x, y: man.gN(TAU, x, y)))
        info = s.step(TAU, tol=1e-12, prec=F.MIXED, inner_tol=1e-2)
        C = s.get_state()
        s.close()
        err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
        assert err <= 1e-9, (persistent, err, info)
        assert info["rel_residual"] <= 1e-12 and info["fp64_iterations"] == 0, (persistent, info)
        out[persistent] = info["iterations"]
    assert abs(out[True] - out[False]) <= max(2, out[False] // 5), out


def test_persistent_switch_is_checked():
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(8, "mixed", seed=3)
    s = gpu_solver(cV, V0T, bdr, 1)
    with pytest.raises(F.FestungError):
        s._check(s.lib.festung_set_persistent(s.h, 2))
    s.close()


def test_persistent_barrier_wait_runs_out_and_is_reported():
    """The bounded waits of the persistent p <= 1 solver: with festung_test_barrier_timeout
    every grid barrier waits for one block more than the grid has, each wait gives up after
    about a second, and the step fails with FESTUNG_ECUDA, leaving the state as it was; the
    context then steps normally and still matches the oracle."""
    import time
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    cV, V0T, bdr = mesh(MESH_N, "mixed", seed=21)
    s = gpu_solver(cV, V0T, bdr, 1)
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    s.set_coeff(samples(s, lambda x, y: man.d(TAU, x, y)))
    s.set_source(samples(s, lambda x, y: man.f(TAU, x, y)))
    s.set_bc(edge_samples(s, lambda x, y: man.c(TAU, x, y)), edge_samples(s, lambda x, y: man.gN(TAU, x, y)))
    C0 = s.get_state()
    s._check(s.lib.festung_test_barrier_timeout(s.h, 1))
    t0 = time.perf_counter()
    with pytest.raises(F.FestungError, match="barrier"):
        s.step(TAU, tol=1e-12, prec=F.MIXED, inner_tol=1e-2)
    assert time.perf_counter() - t0 < 30
    assert np.array_equal(s.get_state(), C0)
    s._check(s.lib.festung_test_barrier_timeout(s.h, 0))
    info = s.step(TAU, tol=1e-12, prec=F.MIXED, inner_tol=1e-2)
    C = s.get_state()
    s.close()
    Co = _oracle(1, "mixed", man, TAU)
    err = np.linalg.norm(C - Co) / np.linalg.norm(Co)
    assert err <= 1e-9, (err, info)
