"""Pins of the oracle's blocks, elimination and solves (Sec. 2.4-2.5, 3.6, 3.9)."""
import os

import numpy as np
import pytest

import workloads as W
from oracle.solve import LDG

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MIXES = {"dirichlet": ((1, 2, 3, 4), ()), "neumann": ((), (1, 2, 3, 4)), "mixed": ((2, 4), (1, 3))}


def _ldg(n, p, mix, jitter=0.2, seed=1, quad_order=None):
    cV, V0T, side = W.square_mesh(n, jitter=jitter, seed=seed)
    dr, nr = MIXES[mix]
    return LDG(cV, V0T, W.boundary_types(side, dr, nr), p, quad_order=quad_order)


def _smooth_d(x, y):
    return 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.3 * x * y


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mix", ["dirichlet", "neumann", "mixed"])
def test_dense_full_system_equals_eliminated(p, mix):
    """Brute force: dense solve of the 3KN system (eq. fullSystem) vs the eliminated solve."""
    L = _ldg(2, p, mix)
    man = W.Manufactured(W.d_config2)
    t, tau = 0.05, 0.01
    D = L.project(lambda x, y: man.d(t, x, y))
    F = L.project(lambda x, y: man.f(t, x, y))
    C0 = L.project(lambda x, y: man.c(0.0, x, y))
    cD = lambda x, y: man.c(t, x, y)
    gN = lambda x, y: man.gN(t, x, y)
    Cd, Z1, Z2 = L.step_full(C0, D, F, cD, gN, tau, dense=True)
    Ce = L.step(C0, D, F, cD, gN, tau)
    assert np.linalg.norm(Cd - Ce) <= 1e-11 * np.linalg.norm(Cd)
    # the flux unknown satisfies z = -M^{-1}(B_m C + J_D^m) (first two block rows)
    from oracle import assemble
    JD = assemble.vec_JD(L.g, L.ref, cD) if L.g.markD.any() else [0 * Cd.ravel()] * 2
    for Z, m in ((Z1, 0), (Z2, 1)):
        Zr = -(L.Minv @ (L.Bm[m] @ Cd.ravel() + JD[m]))
        assert np.linalg.norm(Z.ravel() - Zr) <= 1e-10 * max(1.0, np.linalg.norm(Zr))


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_constant_state_preserved_zero_flux(p):
    """With zero-flux (Neumann) boundaries the constant function is in the kernel of the
    spatial operator: grad c = 0 gives z = 0 and all jumps vanish, so S_op 1 = M 1."""
    L = _ldg(4, p, "neumann")
    D = L.project(_smooth_d)
    one = L.project(lambda x, y: np.ones_like(x))
    y = L.apply(D, 0.1, one)
    Mx = L.M @ one.ravel()
    # rounding scale: the spatial operator's row norm times |x|
    scale = 0.1 * abs(L.operator(D, None)).sum(axis=1).max() * np.abs(one).max()
    assert np.abs(y - Mx).max() <= 1e-13 * scale


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_exact_mass_conservation(p):
    """Testing with w = 1 (the phi_1 row): interior fluxes cancel pairwise because the
    penalty uses 1/|E| (Sec. 2.4.4, S) and the averages are symmetric; with zero-flux
    boundaries the total of the phi_1 rows of the spatial operator vanishes."""
    L = _ldg(4, p, "neumann", seed=7)
    D = L.project(_smooth_d)
    x = np.random.default_rng(p).standard_normal(L.K * L.N)
    r = L.apply(D, 1.0, x) - L.M @ x
    tot = r.reshape(L.K, L.N)[:, 0].sum()
    assert abs(tot) <= 1e-11 * np.abs(r).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetry_iff_elementwise_constant_d(p):
    L = _ldg(3, p, "mixed", seed=5)
    rng = np.random.default_rng(0)
    Dc = np.zeros((L.K, L.N))
    Dc[:, 0] = rng.uniform(0.5, 2.0, L.K)
    S = L.operator(Dc, 0.1).toarray()
    assert np.linalg.norm(S - S.T) <= 1e-13 * np.linalg.norm(S)
    Ds = L.project(_smooth_d)
    S2 = L.operator(Ds, 0.1).toarray()
    assert np.linalg.norm(S2 - S2.T) >= 1e-6 * np.linalg.norm(S2)


def test_verification_rates():
    """Sec. 3.9: L2 errors of the stationary problem converge with order ~ p + 1."""
    gold = {int(p): a for p, a in np.loadtxt(os.path.join(GOLDEN, "verification_rates.txt"))}
    man = W.Manufactured(W.d_verification, stationary=True)
    for p in (1, 2, 3, 4):
        errs = []
        for n in (4, 8, 16):
            cV, V0T, side = W.square_mesh(n)
            L = LDG(cV, V0T, W.boundary_types(side, (2, 4), (1, 3)), p)
            D = L.project(lambda x, y: man.d(0, x, y))
            F = L.project(lambda x, y: man.f(0, x, y))
            C = L.stationary(D, F, lambda x, y: man.c(0, x, y), lambda x, y: man.gN(0, x, y))
            errs.append(L.l2_error(C, lambda x, y: man.c(0, x, y)))
        rate = np.log2(errs[-2] / errs[-1])
        assert abs(rate - (p + 1)) < 0.25, (p, errs, rate, gold[p])


def test_implicit_euler_first_order_in_time():
    cV, V0T, side = W.square_mesh(4)
    L = LDG(cV, V0T, W.boundary_types(side, (1, 2, 3, 4), ()), 2)
    man = W.Manufactured(W.d_config1)
    T = 0.2

    def run(nsteps):
        tau = T / nsteps
        C = L.project(lambda x, y: man.c(0.0, x, y))
        for s in range(1, nsteps + 1):
            t = s * tau
            D = L.project(lambda x, y: man.d(t, x, y))
            F = L.project(lambda x, y: man.f(t, x, y))
            C = L.step(C, D, F, lambda x, y: man.c(t, x, y), None, tau)
        return C

    ref = run(64)
    e = [np.linalg.norm(run(n) - ref) for n in (4, 8, 16)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 1.7 < r1 < 2.6 and 1.7 < r2 < 2.6, e


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("mix", ["dirichlet", "mixed"])
def test_stationary_reproduces_discrete_solutions(p, mix):
    """Consistency (Sec. 2.2-2.4): when c and z = -grad c lie in the discrete space, the
    LDG equations hold for them exactly (jumps vanish, the central fluxes are exact, the
    Neumann flux d g_N is the true one), so the stationary solution is the projection of
    c.  Every block and right-hand-side term enters: a dropped term, a wrong sign or a
    transposed operand breaks it."""
    from helpers import patch_case
    c, d, f, gN = patch_case(p)
    L = _ldg(4, p, mix, seed=5)
    C = L.stationary(L.project(d), L.project(f), c, gN)
    Cp = L.project(c)
    assert np.linalg.norm(C - Cp) <= 1e-11 * np.linalg.norm(Cp)


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("mix", ["dirichlet", "mixed"])
def test_step_reproduces_discrete_solutions_linear_in_time(p, mix):
    """Consistency of the implicit-Euler step (Sec. 2.5): for c(t) = c0 + t c1 with c0,
    c1 and their gradients in the discrete space, the difference quotient of the step is
    exact, so one step from the projection of c(t_n) gives the projection of c(t_n+1)."""
    from helpers import patch_case
    c0, d, f0, gN0 = patch_case(p)
    c1, _, f1, gN1 = patch_case(1)          # a linear rate: its own Laplacian is zero

    def c(t, x, y):
        return c0(x, y) + t * c1(x, y)

    def f(t, x, y):                        # dt c - div(d grad c) = c1 + f0 + t f1
        return c1(x, y) + f0(x, y) + t * f1(x, y)

    def gN(t, x, y):
        return gN0(x, y) + t * gN1(x, y)

    L = _ldg(4, p, mix, seed=5)
    tn, tau = 0.3, 0.05
    t = tn + tau
    C = L.step(L.project(lambda x, y: c(tn, x, y)), L.project(d), L.project(lambda x, y: f(t, x, y)),
               lambda x, y: c(t, x, y), lambda x, y: gN(t, x, y), tau)
    Cp = L.project(lambda x, y: c(t, x, y))
    assert np.linalg.norm(C - Cp) <= 1e-12 * np.linalg.norm(Cp)
