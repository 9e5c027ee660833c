"""What the step's solver would gain from a coarse correction on the low-order modes
(no GPU; the oracle's operator).  After the quadratic extrapolation in time, the error of
the initial guess is smooth in space, which the element-block Jacobi preconditioner
reduces slowly.  The modal basis is hierarchical (Sec. 2.4.1): the p <= 1 coefficients
of every triangle span a coarse space, and a two-level preconditioner (an exact solve of
the Galerkin coarse operator R S R^T, then block Jacobi on the remainder) removes those
components at once.  On a 24 x 24 jittered mesh at p = 3 and tau / h^2 of the 128 x 128
workload, BiCGStab from the extrapolated guess to 1e-10 needs more than ten times fewer
iterations with it."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W


def _bicgstab_iterations(S, b, x0, M, tol):
    count = [0]

    def cb(_):
        count[0] += 1

    x, info = spla.bicgstab(S, b, x0=x0, rtol=tol, atol=0.0, M=spla.LinearOperator(S.shape, matvec=M),
                            callback=cb, maxiter=2000)
    return count[0], np.linalg.norm(b - S @ x) / np.linalg.norm(b)


def _last_step(n, p):
    """Operator, right-hand side and quadratically extrapolated guess of the fifth step."""
    from oracle.solve import LDG
    tau = 16.4 / n ** 2
    cV, V0T, side = W.square_mesh(n, jitter=0.2, seed=11)
    bdr = W.boundary_types(side, (2, 4), (1, 3))
    L = LDG(cV, V0T, bdr, p)
    man = W.Manufactured(W.d_config2)
    K, N = L.K, L.N
    states = [L.project(lambda x, y: man.c(0.0, x, y)).ravel()]
    for k in range(1, 5):
        t = k * tau
        D = L.project(lambda x, y: man.d(t, x, y))
        S = L.operator(D, tau).tocsr()
        b = L.rhs(states[-1].reshape(K, N), D, L.project(lambda x, y: man.f(t, x, y)),
                  lambda x, y: man.c(t, x, y), lambda x, y: man.gN(t, x, y), tau)
        states.append(spla.spsolve(S.tocsc(), b))
    # the last step again, from the quadratic extrapolation through the three states before it
    x0 = 3 * states[-2] - 3 * states[-3] + states[-4]
    return L, D, S, b, x0, cV, V0T, bdr, tau


def test_coarse_correction_cuts_iterations():
    n, p = 24, 3
    L, D, S, b, x0, cV, V0T, bdr, tau = _last_step(n, p)
    K, N = L.K, L.N
    blocks = sp.block_diag([sp.csr_matrix(np.linalg.inv(S[k * N:(k + 1) * N, k * N:(k + 1) * N].toarray()))
                            for k in range(K)]).tocsr()
    coarse = np.concatenate([np.arange(k * N, k * N + 3) for k in range(K)])   # modes of p <= 1
    R = sp.csr_matrix((np.ones(coarse.size), (np.arange(coarse.size), coarse)), shape=(coarse.size, K * N))
    lu = spla.splu((R @ S @ R.T).tocsc())

    def block_jacobi(r):
        return blocks @ r

    def two_level(r):
        e = R.T @ lu.solve(R @ r)
        return e + blocks @ (r - S @ e)

    it_bj, rr_bj = _bicgstab_iterations(S, b, x0, block_jacobi, 1e-10)
    it_2l, rr_2l = _bicgstab_iterations(S, b, x0, two_level, 1e-10)
    assert rr_bj <= 2e-10 and rr_2l <= 2e-10
    assert 10 * it_2l <= it_bj, (it_bj, it_2l)


def test_one_shot_rediscretised_coarse_correction():
    """The form the library uses (festung_set_coarse): before a block-Jacobi sweep, solve the
    p = 1 problem on the same mesh (d_h replaced by its P1 part, the same tau) for the P1
    part of the residual, only to 1e-2, and start the sweep from that correction.  The error
    it acts on is the smooth remainder that block-Jacobi BiCGStab leaves behind (here: what
    is left after a 1e3-fold reduction from C^n, as the extrapolated guesses of the bench
    workload leave); a sweep that reduces the residual 20-fold then needs several times
    fewer iterations."""
    from oracle.solve import LDG
    n, p, tau = 40, 3, 1e-3
    cV, V0T, side = W.square_mesh(n, jitter=0.2, seed=11)
    bdr = W.boundary_types(side, (2, 4), (1, 3))
    man = W.Manufactured(W.d_config2)
    L = LDG(cV, V0T, bdr, p)
    K, N = L.K, L.N
    t1 = 0.5 + tau
    D = L.project(lambda x, y: man.d(t1, x, y))
    S = L.operator(D, tau).tocsr()
    xs = L.project(lambda x, y: man.c(t1, x, y)).ravel()
    b = S @ xs
    blocks = sp.block_diag([sp.csr_matrix(np.linalg.inv(S[k * N:(k + 1) * N, k * N:(k + 1) * N].toarray()))
                            for k in range(K)]).tocsr()
    bj = spla.LinearOperator(S.shape, matvec=lambda v: blocks @ v)
    xc = L.project(lambda x, y: man.c(0.5, x, y)).ravel()
    r_c = np.linalg.norm(b - S @ xc) / np.linalg.norm(b)
    x0, _ = spla.bicgstab(S, b, x0=xc, rtol=1e-3 * r_c, atol=0.0, M=bj, maxiter=5000)
    L1 = LDG(cV, V0T, bdr, 1)
    S1 = L1.operator(D[:, :3], tau).tocsr()
    blocks1 = sp.block_diag([sp.csr_matrix(np.linalg.inv(S1[k * 3:(k + 1) * 3, k * 3:(k + 1) * 3].toarray()))
                             for k in range(K)]).tocsr()
    coarse = np.concatenate([np.arange(k * N, k * N + 3) for k in range(K)])
    r = b - S @ x0
    d1, _ = spla.bicgstab(S1, r[coarse], rtol=1e-2, atol=0.0,
                          M=spla.LinearOperator(S1.shape, matvec=lambda v: blocks1 @ v), maxiter=2000)
    x1 = x0.copy()
    x1[coarse] += d1
    target = 0.05 * np.linalg.norm(r) / np.linalg.norm(b)
    it_0, rr_0 = _bicgstab_iterations(S, b, x0, lambda v: blocks @ v, target)
    it_1, rr_1 = _bicgstab_iterations(S, b, x1, lambda v: blocks @ v, target)
    assert rr_0 <= 1.01 * target and rr_1 <= 1.01 * target
    assert 3 * it_1 <= it_0, (it_0, it_1)
