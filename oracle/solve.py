"""The implicit-Euler system (Sec. 2.5, eq. fullSystem) and its solution.

One step of the paper (Sec. 2.5) solves, for Y = [Z^1; Z^2; C],

    (W + tau A(t^{n+1})) Y^{n+1} = W Y^n + tau V(t^{n+1})                 (*)

with A and V of eq. timeDepSystem:

    A = [ M    0    -H^1 + Q^1 + Q_N^1 ]      V = [ -J_D^1                 ]
        [ 0    M    -H^2 + Q^2 + Q_N^2 ]          [ -J_D^2                 ]
        [ A_1  A_2  eta (S + S_D)      ]          [ eta K_D - K_N + L      ]

    A_m = -G^m + R^m + R_D^m,  W = diag(0, 0, M).

``step_full`` assembles (*) exactly like the paper's main script and solves it with a
sparse direct solver (SuperLU).  The first two block rows give
Z^m = -M^{-1} (B_m C + J_D^m) with B_m = -H^m + Q^m + Q_N^m; inserting this in the
third row gives the step operator on C alone,

    S_op C = M C + tau (eta (S + S_D) C - sum_m A_m M^{-1} B_m C)
    b      = M C^n + tau (eta K_D - K_N + L + sum_m A_m M^{-1} J_D^m),

which ``operator`` and ``rhs`` form explicitly (CSR); ``apply`` is S_op x.  The
stationary problem of Sec. 3.9 drops M and tau:
(eta (S + S_D) - sum_m A_m M^{-1} B_m) C = eta K_D - K_N + L + sum_m A_m M^{-1} J_D^m.

Parity: pinned (dense 3KN solve equals the eliminated solve on small meshes; constant
states preserved; exact conservation; symmetry for elementwise-constant d; L2
convergence rates p + 1 on the problem of Sec. 3.9; first-order convergence in tau).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble, basis, grid, project, quadrature, reference


class LDG:
    """Discretisation of Sec. 2 on one mesh for one order p."""

    def __init__(self, coordV, V0T, bdr, p, quad_order=None, eta=1.0):
        if not 0 <= p <= basis.PMAX:
            raise ValueError("p must be in 0..4")
        self.p = p
        self.N = basis.num_dofs(p)
        self.qT = max(1, 2 * p if quad_order is None else int(quad_order))
        self.qE = max(self.qT, 2 * p + 1)
        self.R1 = quadrature.edge_points_for_degree(self.qE)
        self.eta = float(eta)
        self.g = grid.generate_grid_data(coordV, V0T, bdr)
        self.ref = reference.compute(p, self.qT, self.R1)
        g, ref = self.g, self.ref
        self.M = assemble.mass(g, ref)
        self.Minv = sp.diags(1.0 / self.M.diagonal())
        H = assemble.mat_H(g, ref)
        Q = assemble.mat_Q(g, ref)
        QN = assemble.mat_QN(g, ref)
        self.Bm = [(-H[m] + Q[m] + QN[m]).tocsr() for m in range(2)]
        self.St = (assemble.mat_S(g, ref) + assemble.mat_SD(g, ref)).tocsr()

    # ----- data ---------------------------------------------------------------
    @property
    def K(self):
        return self.g.numT

    def project(self, func):
        return project.project(self.g, func, self.N, self.qT)

    def project_samples(self, samples):
        return project.project_samples(samples, self.N, self.qT)

    def quad_points(self):
        q1, q2, _ = quadrature.triangle_rule(self.qT)
        return grid.map_to_physical(self.g, q1, q2)

    def edge_points(self):
        """Physical Gauss points [K, 3, R1] (x, y) of every local edge."""
        s, _ = self.ref.edge
        X = np.zeros((self.K, 3, self.R1))
        Y = np.zeros((self.K, 3, self.R1))
        for n in range(3):
            x1, x2 = quadrature.gamma_map(n, s)
            X[:, n], Y[:, n] = grid.map_to_physical(self.g, x1, x2)
        return X, Y

    # ----- time-dependent blocks -----------------------------------------------
    def Am(self, D):
        g, ref = self.g, self.ref
        G = assemble.mat_G(g, ref, D)
        R = assemble.mat_R(g, ref, D)
        RD = assemble.mat_RD(g, ref, D)
        return [(-G[m] + R[m] + RD[m]).tocsr() for m in range(2)]

    def operator(self, D, tau):
        """Step operator S_op (CSR); tau = None gives the stationary operator."""
        A = self.Am(D)
        coupling = A[0] @ self.Minv @ self.Bm[0] + A[1] @ self.Minv @ self.Bm[1]
        L = self.eta * self.St - coupling
        if tau is None:
            return L.tocsr()
        return (self.M + tau * L).tocsr()

    def rhs(self, C_old, D, F, cD, gN, tau):
        """b of the eliminated step (tau = None: stationary right-hand side)."""
        g, ref = self.g, self.ref
        A = self.Am(D)
        v = np.zeros(self.K * self.N)
        if g.markD.any():
            JD = assemble.vec_JD(g, ref, cD)
            v += self.eta * assemble.vec_KD(g, ref, cD)
            v += A[0] @ (self.Minv @ JD[0]) + A[1] @ (self.Minv @ JD[1])
        if g.markN.any() and gN is not None:
            v -= assemble.vec_KN(g, ref, D, gN)
        if F is not None:
            v += assemble.vec_L(g, ref, F)
        if tau is None:
            return v
        return self.M @ np.asarray(C_old).ravel() + tau * v

    def apply(self, D, tau, x):
        return self.operator(D, tau) @ np.asarray(x).ravel()

    # ----- solves ----------------------------------------------------------------
    def step(self, C_old, D, F, cD, gN, tau):
        """C^{n+1} from the eliminated system (sparse direct)."""
        S = self.operator(D, tau).tocsc()
        b = self.rhs(C_old, D, F, cD, gN, tau)
        return spla.spsolve(S, b).reshape(self.K, self.N)

    def full_system(self, C_old, D, F, cD, gN, tau):
        """(W + tau A, W Y^n + tau V) of eq. fullSystem, Y = [Z^1; Z^2; C]."""
        g, ref = self.g, self.ref
        KN = self.K * self.N
        A = self.Am(D)
        Z = sp.csr_matrix((KN, KN))
        Amat = sp.bmat([[self.M, Z, self.Bm[0]],
                        [Z, self.M, self.Bm[1]],
                        [A[0], A[1], self.eta * self.St]]).tocsr()
        W = sp.bmat([[Z, Z, Z], [Z, Z, Z], [Z, Z, self.M]]).tocsr()
        V = np.zeros(3 * KN)
        if g.markD.any():
            JD = assemble.vec_JD(g, ref, cD)
            V[:KN] = -JD[0]
            V[KN:2 * KN] = -JD[1]
            V[2 * KN:] += self.eta * assemble.vec_KD(g, ref, cD)
        if g.markN.any() and gN is not None:
            V[2 * KN:] -= assemble.vec_KN(g, ref, D, gN)
        if F is not None:
            V[2 * KN:] += assemble.vec_L(g, ref, F)
        Yold = np.zeros(3 * KN)
        Yold[2 * KN:] = np.asarray(C_old).ravel()
        return (W + tau * Amat).tocsc(), W @ Yold + tau * V

    def step_full(self, C_old, D, F, cD, gN, tau, dense=False):
        """Solve eq. fullSystem for one step as the paper's main script does."""
        Amat, v = self.full_system(C_old, D, F, cD, gN, tau)
        if dense:
            Y = np.linalg.solve(Amat.toarray(), v)
        else:
            Y = spla.spsolve(Amat, v)
        KN = self.K * self.N
        return (Y[2 * KN:].reshape(self.K, self.N),
                Y[:KN].reshape(self.K, self.N), Y[KN:2 * KN].reshape(self.K, self.N))

    def stationary(self, D, F, cD, gN):
        S = self.operator(D, None).tocsc()
        b = self.rhs(None, D, F, cD, gN, None)
        return spla.spsolve(S, b).reshape(self.K, self.N)

    def l2_error(self, C, func, qT=None):
        return project.l2_error(self.g, C, func, 2 * self.p + 2 if qT is None else qT)
