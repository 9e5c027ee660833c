"""L2 projection (Sec. 3.4, routine projectFuncCont2DataDisc) and the discretisation
error (Sec. 3.5, routine computeL2Error).

Projection: D M^ = sum_r w_r d(F_k(q_r)) phi_j(q_r), solved with M^ (= I here, Sec. 2.4.1).
L2 error:   ||c_h - c||^2 = 2 sum_k |T_k| sum_r w_r (sum_l C_kl phi_l(q_r) - c(F_k(q_r)))^2.

Parity: pinned (polynomials of degree <= p are reproduced; the two-triangle example of
Sec. 3.10 reproduces the printed value ranges).
"""
import numpy as np

from . import basis, quadrature
from .grid import map_to_physical


def project(g, func, N, qT):
    """[K, N] representation matrix of the L2 projection of func(x1, x2) (arrays [K, R])."""
    q1, q2, w = quadrature.triangle_rule(qT)
    X, Y = map_to_physical(g, q1, q2)
    vals = func(X, Y)                                  # [K, R]
    rhs = vals @ (w[:, None] * basis.phi_table(N, q1, q2))
    hatM = np.eye(N)
    return np.linalg.solve(hatM, rhs.T).T


def project_samples(samples, N, qT):
    """Same projection from samples already taken at the physical quadrature points [K, R]."""
    q1, q2, w = quadrature.triangle_rule(qT)
    return np.asarray(samples) @ (w[:, None] * basis.phi_table(N, q1, q2))


def l2_error(g, C, func, qT):
    q1, q2, w = quadrature.triangle_rule(qT)
    X, Y = map_to_physical(g, q1, q2)
    N = C.shape[1]
    ch = C @ basis.phi_table(N, q1, q2).T              # [K, R]
    err2 = 2.0 * np.dot(((ch - func(X, Y)) ** 2) @ w, g.areaT)
    return float(np.sqrt(err2))


def evaluate(C, x1, x2):
    """c_h at reference points (x1, x2) in every element: [K, R]."""
    N = C.shape[1]
    return C @ basis.phi_table(N, x1, x2).T
