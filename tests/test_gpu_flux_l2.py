"""Flux recovery and L2 error on the GPU (festung_get_flux, festung_l2_error).

Z^m = -M^{-1} (B_m C + J_D^m) are block rows 1-2 of eq. timeDepSystem: the oracle's
solve of the full 3KN system (eq. fullSystem) returns them next to C.  A linear c with
its own Dirichlet data has the exact discrete gradient (z_h = -grad c, Sec. 2.2).  The
L2 error of Sec. 3.5 is compared with the oracle's evaluation under the same triangle rule.
"""
import numpy as np
import pytest

import workloads as W
from helpers import edge_samples, gpu_solver, mesh, samples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mix", ["dirichlet", "mixed"])
def test_flux_matches_full_system(p, mix):
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(6, mix, seed=3)
    man = W.Manufactured(W.d_config2)
    tau, t = 0.01, 0.01
    L = LDG(cV, V0T, bdr, p)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    s.set_coeff(samples(s, lambda x, y: man.d(t, x, y)))
    s.set_source(samples(s, lambda x, y: man.f(t, x, y)))
    s.set_bc(edge_samples(s, lambda x, y: man.c(t, x, y)), edge_samples(s, lambda x, y: man.gN(t, x, y)))
    s.step(tau, tol=1e-13, prec=F.FP64)
    Z = s.get_flux()
    C0 = L.project(lambda x, y: man.c(0.0, x, y))
    _, Z1, Z2 = L.step_full(C0, L.project(lambda x, y: man.d(t, x, y)), L.project(lambda x, y: man.f(t, x, y)),
                            lambda x, y: man.c(t, x, y), lambda x, y: man.gN(t, x, y), tau)
    for got, want in ((Z[0], Z1), (Z[1], Z2)):
        assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(np.stack([Z1, Z2])), \
            np.linalg.norm(got - want) / np.linalg.norm(want)
    s.close()


@pytest.mark.parametrize("p", [1, 2, 4])
def test_flux_of_linear_function_is_exact(p):
    cV, V0T, bdr = mesh(5, "dirichlet", seed=4)
    a, b, c = 0.3, -1.7, 2.2
    lin = lambda x, y: a + b * x + c * y
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_bc(edge_samples(s, lin), None)
    s.set_state(samples(s, lambda x, y: 0 * x - b), is_samples=True)
    want1 = s.get_state()                       # projection of the constant -b
    s.set_state(samples(s, lambda x, y: 0 * x - c), is_samples=True)
    want2 = s.get_state()
    s.set_state(samples(s, lin), is_samples=True)
    Z = s.get_flux()
    assert np.max(np.abs(Z[0] - want1)) <= 1e-12 * abs(b) * 10
    assert np.max(np.abs(Z[1] - want2)) <= 1e-12 * abs(c) * 10
    s.close()


@pytest.mark.parametrize("p", [1, 2])
def test_l2_error_matches_oracle_rule(p):
    from oracle.solve import LDG
    cV, V0T, bdr = mesh(7, "mixed", seed=5)
    f = lambda x, y: np.exp(x) * np.sin(3 * y)
    L = LDG(cV, V0T, bdr, p)
    s = gpu_solver(cV, V0T, bdr, p)
    C = L.project(lambda x, y: np.cos(2 * x) * y)  # some state, not the projection of f
    s.set_state(C, is_samples=False)
    got = s.l2_error(samples(s, f))
    want = L.l2_error(C, f, qT=2 * p)
    assert abs(got - want) <= 1e-12 * want, (got, want)
    # polynomials of degree <= p are reproduced: zero error
    poly = lambda x, y: 1.0 + x - 2 * y + (0.5 * x * y if p >= 2 else 0.0)
    s.set_state(samples(s, poly), is_samples=True)
    assert s.l2_error(samples(s, poly)) <= 1e-13
    s.close()
