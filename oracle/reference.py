"""Reference-element integrals (Sec. 3.6.1-3.6.6, routines integrateRef*).

All arrays follow the paper's index order (0-based):

  hatM[i, j]                  = int_T^ phi_i phi_j                         (eq. hatM) = I
  hatH[i, j, m]               = int_T^ d_m phi_i phi_j                     (eq. hatH)
  hatG[i, j, l, m]            = int_T^ d_m phi_i phi_j phi_l               (eq. hatG)
  hatSdiag[i, j, n]           = int_0^1 phi_i(g_n(s)) phi_j(g_n(s)) ds     (eq. hatSdiag)
  hatSoffdiag[i, j, n-, n+]   = int_0^1 phi_i(g_n-(s)) phi_j(th(g_n-(s)))  (eq. hatSoffdiag)
  hatRdiag[i, j, l, n]        = int_0^1 phi_i phi_l phi_j on g_n           (eq. hatRdiag)
  hatRoffdiag[i, j, l, n-, n+]= int_0^1 phi_i(g) phi_l(th(g)) phi_j(th(g))  (eq. hatRoffdiag)

with g_n the edge parametrisation (eq. gammaMap) and th the edge-to-edge maps
(eq. mapEE).  Volume integrals use the triangle rule of degree ``qT`` and edge
integrals the Gauss rule with ``R1`` points, exactly as the paper evaluates them by
quadrature (Sec. 3.3: degree 2p on triangles and 2p + 1 on edges by default).
M^ is the identity by orthonormality (Sec. 2.4.1) and is returned as such.

Parity: pinned through the operator-level tests (dense system, conservation,
symmetry, convergence rates).
"""
import numpy as np

from . import basis, quadrature


class RefTensors:
    pass


def compute(p, qT, R1):
    N = basis.num_dofs(p)
    ref = RefTensors()
    ref.p, ref.N, ref.qT, ref.R1 = p, N, qT, R1
    q1, q2, w = quadrature.triangle_rule(qT)
    s, ws = quadrature.gauss_legendre_01(R1)
    ref.tri = (q1, q2, w)
    ref.edge = (s, ws)
    phi = basis.phi_table(N, q1, q2)            # [R2, N]
    gphi = basis.grad_phi_table(N, q1, q2)      # [R2, N, 2]
    ref.hatM = np.eye(N)
    ref.hatH = np.einsum("r,rim,rj->ijm", w, gphi, phi)
    ref.hatG = np.einsum("r,rim,rj,rl->ijlm", w, gphi, phi, phi)

    phi1 = np.zeros((R1, N, 3))                 # phi_i(g_n(s_r))
    thphi1 = np.zeros((R1, N, 3, 3))            # phi_i(th_{n-n+}(g_{n-}(s_r)))
    for nm in range(3):
        x1, x2 = quadrature.gamma_map(nm, s)
        phi1[:, :, nm] = basis.phi_table(N, x1, x2)
        for npl in range(3):
            y1, y2 = quadrature.theta_map(nm, npl, x1, x2)
            thphi1[:, :, nm, npl] = basis.phi_table(N, y1, y2)
    ref.phi1, ref.thphi1 = phi1, thphi1
    ref.hatSdiag = np.einsum("r,rin,rjn->ijn", ws, phi1, phi1)
    ref.hatSoffdiag = np.einsum("r,rin,rjnp->ijnp", ws, phi1, thphi1)
    ref.hatRdiag = np.einsum("r,rin,rln,rjn->ijln", ws, phi1, phi1, phi1)
    ref.hatRoffdiag = np.einsum("r,rin,rlnp,rjnp->ijlnp", ws, phi1, thphi1, thphi1)
    return ref
