"""Global block matrices and right-hand-side vectors (Sec. 2.4.3-2.4.4 and 3.6).

Each function returns a scipy.sparse CSR matrix of size KN x KN (or a length-KN
vector) in the paper's global ordering (k - 1) N + i (0-based: k N + i).  The
block definitions follow Sec. 3.6 term by term:

  M      = 2 diag(|T_k|) (x) M^                                   (Sec. 3.6.1)
  H^m    = B-weighted Kronecker products of H^                      (Sec. 3.6.2)
  G^m    = sum_l D_kl (B-weighted G^[:, :, l, :])                  (Sec. 3.6.3)
  S      = S^diag on interior edges - markE0TE0T (x) S^offdiag      (Sec. 3.6.4, eq. globS)
  Q^m    = 1/2 nu^m |E| (S^diag, S^offdiag) on interior edges       (Sec. 3.6.5, eq. globQ)
  R^m    = 1/2 nu^m |E| sum_l D (R^diag, R^offdiag)                 (Sec. 3.6.6, eq. globR)
  R_D^m, S_D, Q_N^m: the diagonal parts on Dirichlet / Dirichlet / Neumann edges
                                                                    (Sec. 3.6.7-3.6.9)
  J_D^m, K_D, K_N, L: right-hand sides                              (Sec. 3.6.10-3.6.12)

For the diagonal part of R^2 the equation (eq. globR:diag, nu^2) is followed.

Parity: pinned through the dense-system, conservation, symmetry and convergence
tests.
"""
import numpy as np
import scipy.sparse as sp

from . import basis, quadrature
from .grid import map_to_physical


def _blocks_to_csr(K, N, rows, cols, blocks):
    """Sum of N x N blocks placed at block positions (rows[t], cols[t])."""
    if len(rows) == 0:
        return sp.csr_matrix((K * N, K * N))
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    blocks = np.asarray(blocks, dtype=np.float64)
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    R = (rows[:, None, None] * N + ii[None]).ravel()
    C = (cols[:, None, None] * N + jj[None]).ravel()
    return sp.coo_matrix((blocks.ravel(), (R, C)), shape=(K * N, K * N)).tocsr()


def _diag_blocks(K, N, blocks):
    k = np.arange(K)
    return _blocks_to_csr(K, N, k, k, blocks)


def mass(g, ref):
    K, N = g.numT, ref.N
    return _diag_blocks(K, N, 2.0 * g.areaT[:, None, None] * ref.hatM[None])


def _bweights(g, m):
    """Coefficients (c1, c2) with d_{x^m} = (c1 d_x^1 + c2 d_x^2) / (2|T|), eq. rule:gradient."""
    B = g.B
    if m == 0:
        return B[:, 1, 1], -B[:, 1, 0]
    return -B[:, 0, 1], B[:, 0, 0]


def mat_H(g, ref):
    K, N = g.numT, ref.N
    out = []
    for m in range(2):
        c1, c2 = _bweights(g, m)
        blk = c1[:, None, None] * ref.hatH[None, :, :, 0] + c2[:, None, None] * ref.hatH[None, :, :, 1]
        out.append(_diag_blocks(K, N, blk))
    return out


def mat_G(g, ref, D):
    K, N = g.numT, ref.N
    out = []
    for m in range(2):
        c1, c2 = _bweights(g, m)
        GD0 = np.einsum("kl,ijl->kij", D, ref.hatG[:, :, :, 0])
        GD1 = np.einsum("kl,ijl->kij", D, ref.hatG[:, :, :, 1])
        blk = c1[:, None, None] * GD0 + c2[:, None, None] * GD1
        out.append(_diag_blocks(K, N, blk))
    return out


def _edge_diag(g, ref, mark, weight_kn):
    """sum_n mark[k, n] * weight_kn[k, n] * S^diag[:, :, n] as diagonal blocks."""
    K, N = g.numT, ref.N
    blk = np.einsum("kn,ijn->kij", mark * weight_kn, ref.hatSdiag)
    return _diag_blocks(K, N, blk)


def _offdiag_pairs(g):
    rows, cols, nms, nps = [], [], [], []
    for (nm, npl), pairs in g.markE0TE0T.items():
        for (km, kp) in pairs:
            rows.append(km)
            cols.append(kp)
            nms.append(nm)
            nps.append(npl)
    return (np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64),
            np.array(nms, dtype=np.int64), np.array(nps, dtype=np.int64))


def mat_S(g, ref):
    """Penalty matrix S without the factor eta (eq. globS); edge lengths cancel."""
    K, N = g.numT, ref.N
    diag = _edge_diag(g, ref, g.markInt.astype(float), np.ones((K, 3)))
    r, c, nm, npl = _offdiag_pairs(g)
    off = _blocks_to_csr(K, N, r, c, -ref.hatSoffdiag[:, :, nm, npl].transpose(2, 0, 1))
    return diag + off


def mat_SD(g, ref):
    return _edge_diag(g, ref, g.markD.astype(float), np.ones((g.numT, 3)))


def mat_Q(g, ref):
    K, N = g.numT, ref.N
    r, c, nm, npl = _offdiag_pairs(g)
    out = []
    for m in range(2):
        wkn = 0.5 * g.nuE0T[:, :, m] * g.areaE0T
        diag = _edge_diag(g, ref, g.markInt.astype(float), wkn)
        offblk = (wkn[r, nm])[:, None, None] * ref.hatSoffdiag[:, :, nm, npl].transpose(2, 0, 1)
        out.append(diag + _blocks_to_csr(K, N, r, c, offblk))
    return out


def mat_QN(g, ref):
    out = []
    for m in range(2):
        wkn = g.nuE0T[:, :, m] * g.areaE0T
        out.append(_edge_diag(g, ref, g.markN.astype(float), wkn))
    return out


def _rdiag_blocks(g, ref, D, mark, wkn):
    # sum_n mark w_kn sum_l D_kl R^diag[:, :, l, n]
    RD = np.einsum("kl,ijln->knij", D, ref.hatRdiag)
    return np.einsum("kn,knij->kij", mark * wkn, RD)


def mat_R(g, ref, D):
    K, N = g.numT, ref.N
    r, c, nm, npl = _offdiag_pairs(g)
    out = []
    for m in range(2):
        wkn = 0.5 * g.nuE0T[:, :, m] * g.areaE0T
        diag = _diag_blocks(K, N, _rdiag_blocks(g, ref, D, g.markInt.astype(float), wkn))
        # off-diagonal: 1/2 nu^m_{k-n-} |E| sum_l D_{k+ l} R^offdiag[:, :, l, n-, n+]
        offblk = np.einsum("tl,ijlt->tij", D[c], ref.hatRoffdiag[:, :, :, nm, npl])
        offblk = wkn[r, nm][:, None, None] * offblk
        out.append(diag + _blocks_to_csr(K, N, r, c, offblk))
    return out


def mat_RD(g, ref, D):
    K, N = g.numT, ref.N
    out = []
    for m in range(2):
        wkn = g.nuE0T[:, :, m] * g.areaE0T
        out.append(_diag_blocks(K, N, _rdiag_blocks(g, ref, D, g.markD.astype(float), wkn)))
    return out


def _edge_function_values(g, ref, func, n):
    """func at the physical Gauss points of local edge n of every triangle: [K, R1]."""
    s, _ = ref.edge
    x1, x2 = quadrature.gamma_map(n, s)
    X, Y = map_to_physical(g, x1, x2)
    return func(X, Y)


def vec_JD(g, ref, cD):
    """J_D^m (Sec. 3.6.10): sum_{n in D} nu^m |E| sum_r w_r phi_i(g_n(s_r)) c_D."""
    K, N = g.numT, ref.N
    _, ws = ref.edge
    out = [np.zeros((K, N)), np.zeros((K, N))]
    for n in range(3):
        if not g.markD[:, n].any():
            continue
        vals = _edge_function_values(g, ref, cD, n)          # [K, R1]
        integ = (vals * ws[None, :]) @ ref.phi1[:, :, n]    # [K, N]
        for m in range(2):
            out[m] += (g.markD[:, n] * g.nuE0T[:, n, m] * g.areaE0T[:, n])[:, None] * integ
    return [o.ravel() for o in out]


def vec_KD(g, ref, cD):
    """K_D (Sec. 3.6.11): edge length cancels against the 1/|E| penalty scaling."""
    K, N = g.numT, ref.N
    _, ws = ref.edge
    out = np.zeros((K, N))
    for n in range(3):
        if not g.markD[:, n].any():
            continue
        vals = _edge_function_values(g, ref, cD, n)
        out += g.markD[:, n][:, None] * ((vals * ws[None, :]) @ ref.phi1[:, :, n])
    return out.ravel()


def vec_KN(g, ref, D, gN):
    """K_N (Sec. 3.6.12): sum_{n in N} |E| sum_l D_kl sum_r w_r phi_i phi_l g_N."""
    K, N = g.numT, ref.N
    _, ws = ref.edge
    out = np.zeros((K, N))
    for n in range(3):
        if not g.markN[:, n].any():
            continue
        vals = _edge_function_values(g, ref, gN, n)                  # [K, R1]
        dtrace = D @ ref.phi1[:, :, n].T                              # [K, R1]
        out += (g.markN[:, n] * g.areaE0T[:, n])[:, None] * ((vals * dtrace * ws[None, :]) @ ref.phi1[:, :, n])
    return out.ravel()


def vec_L(g, ref, F):
    """L = M F (Sec. 2.4.3, term VII)."""
    return mass(g, ref) @ np.asarray(F).ravel()
