"""Reuse of the block-Jacobi blocks over time steps (festung_set_precond_reuse).

The preconditioner does not enter the answer: a trajectory whose steps reuse the blocks of
an earlier step (a lagged preconditioner: d_h changes with t) reaches the same states,
within the solve tolerance, as one that builds them every step, and the schedule of builds
follows the reuse bound, a change of dt and the iteration-growth rule."""
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


def _trajectory(p, reuse, prec, dts, coarse=False, tol=1e-12):
    from paper_1408_3877_gb300 import festung as F
    man = W.Manufactured(W.d_config2)
    cV, V0T, bdr = mesh(MESH_N, "mixed", seed=21)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_precond_reuse(reuse)
    if coarse:
        s.set_coarse(True)
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    t, infos = 0.0, []
    for dt in dts:
        t += dt
        s.set_coeff(samples(s, lambda x, y: man.d(t, x, y)))
        s.set_source(samples(s, lambda x, y: man.f(t, x, y)))
        s.set_bc(edge_samples(s, lambda x, y: man.c(t, x, y)), edge_samples(s, lambda x, y: man.gN(t, x, y)))
        kw = {} if prec == F.FP64 else {"inner_tol": 1e-2}
        infos.append(s.step(dt, tol=tol, prec=prec, **kw))
    C = s.get_state()
    s.close()
    return C, infos


@pytest.mark.parametrize("prec_name,coarse", [("FP64", False), ("MIXED", False), ("MIXED", True)])
def test_reused_blocks_give_the_same_trajectory(prec_name, coarse):
    from paper_1408_3877_gb300 import festung as F
    prec = getattr(F, prec_name)
    dts = [TAU] * 5
    C1, i1 = _trajectory(3, 1, prec, dts, coarse)
    C4, i4 = _trajectory(3, 4, prec, dts, coarse)
    assert [i["precond_built"] for i in i1] == [1] * 5
    built = [i["precond_built"] for i in i4]
    assert built[0] == 1 and built[4] == 1 and built[1:4] == [0, 0, 0], (built, i4)
    for i in i1 + i4:
        assert i["rel_residual"] <= 1e-12, i
    err = np.linalg.norm(C4 - C1) / np.linalg.norm(C1)
    assert err <= 1e-9, err


def test_a_new_dt_rebuilds():
    from paper_1408_3877_gb300 import festung as F
    _, infos = _trajectory(2, 8, F.MIXED, [TAU, TAU, 2 * TAU, 2 * TAU, TAU])
    assert [i["precond_built"] for i in infos] == [1, 0, 1, 0, 1], infos


def test_reuse_bound_is_checked():
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(8, "mixed", seed=3)
    s = gpu_solver(cV, V0T, bdr, 1)
    with pytest.raises(F.FestungError):
        s.set_precond_reuse(0)
    s.close()
