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


def test_coarse_correction_cuts_iterations():
    from oracle.solve import LDG
    n, p = 24, 3
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
