"""Grid lists of Tab. 1 (Sec. 3.1, routine generateGridData), 0-based.

Input: vertex coordinates coordV [numV, 2], counter-clockwise triangles V0T [K, 3],
and per local edge a boundary type bdr [K, 3] (0 interior, 1 Dirichlet, 2 Neumann).
Local edge n of T_k lies opposite vertex n, i.e. runs from a_{k,n+1} to a_{k,n+2}
(indices mod 3), which is the orientation of the edge parametrisation gamma^_n
(eq. gammaMap).

Lists produced (paper names):
  B [K, 2, 2]        B_k = [a_k2 - a_k1 | a_k3 - a_k1]  (eq. affinemappings)
  areaT [K]          |T_k| = det(B_k) / 2
  E0T [K, 3]         global edge index of local edge n
  T0E [numE, 2]      the two triangles of an edge (second = -1 on the boundary)
  E0E [numE, 2]      local edge index of the edge in T0E[:, 0] / T0E[:, 1]
  areaE0T [K, 3]     |E_kn|
  nuE0T [K, 3, 2]    unit normal of E_kn exterior to T_k
  markE0TE0T         dict (n-, n+) -> list of (k-, k+) with E_{k- n-} = E_{k+ n+}
  coordV0T [K, 3, 2] vertex coordinates a_kn

Parity: pinned (closed-triangle identity sum_n |E_kn| nu_kn = 0, outward normals,
edge count, two-triangle example of Sec. 3.10, matching of shared edges).
"""
import numpy as np


class Grid:
    pass


def generate_grid_data(coordV, V0T, bdr):
    coordV = np.asarray(coordV, dtype=np.float64)
    V0T = np.asarray(V0T, dtype=np.int64)
    bdr = np.asarray(bdr, dtype=np.int64)
    K = V0T.shape[0]
    g = Grid()
    g.coordV, g.V0T, g.numT, g.numV = coordV, V0T, K, coordV.shape[0]
    g.coordV0T = coordV[V0T]                              # [K, 3, 2]
    a1, a2, a3 = g.coordV0T[:, 0], g.coordV0T[:, 1], g.coordV0T[:, 2]
    g.B = np.stack([a2 - a1, a3 - a1], axis=-1)           # B[k, m, col]
    g.areaT = 0.5 * (g.B[:, 0, 0] * g.B[:, 1, 1] - g.B[:, 0, 1] * g.B[:, 1, 0])
    if np.any(g.areaT <= 0):
        raise ValueError("triangles must be counter-clockwise and non-degenerate")

    # local edge n runs from vertex n+1 to vertex n+2 (mod 3)
    va = V0T[:, [1, 2, 0]]
    vb = V0T[:, [2, 0, 1]]
    vec = g.coordV[vb] - g.coordV[va]                     # [K, 3, 2] edge vectors (CCW)
    g.areaE0T = np.sqrt(vec[..., 0] ** 2 + vec[..., 1] ** 2)
    # exterior normal of a counter-clockwise edge: rotate its direction by -pi/2
    g.nuE0T = np.stack([vec[..., 1], -vec[..., 0]], axis=-1) / g.areaE0T[..., None]

    # global edge numbering by sorted vertex pairs
    lo = np.minimum(va, vb).ravel()
    hi = np.maximum(va, vb).ravel()
    key = lo * g.numV + hi
    uniq, inv, counts = np.unique(key, return_inverse=True, return_counts=True)
    if np.any(counts > 2):
        raise ValueError("non-manifold edge")
    g.numE = uniq.size
    g.E0T = inv.reshape(K, 3)
    g.T0E = -np.ones((g.numE, 2), dtype=np.int64)
    g.E0E = -np.ones((g.numE, 2), dtype=np.int64)
    for k in range(K):
        for n in range(3):
            e = g.E0T[k, n]
            slot = 0 if g.T0E[e, 0] < 0 else 1
            g.T0E[e, slot] = k
            g.E0E[e, slot] = n

    interior = g.T0E[:, 1] >= 0
    g.bdr = bdr.copy()
    for k in range(K):
        for n in range(3):
            e = g.E0T[k, n]
            if interior[e] and bdr[k, n] != 0:
                raise ValueError("interior edge marked as boundary")
            if not interior[e] and bdr[k, n] == 0:
                raise ValueError("boundary edge without a boundary type")
    g.markInt = bdr == 0
    g.markD = bdr == 1
    g.markN = bdr == 2

    # markE0TE0T{n-, n+}: pairs (k-, k+) sharing an interior edge
    g.markE0TE0T = {(a, b): [] for a in range(3) for b in range(3)}
    for e in np.nonzero(interior)[0]:
        k0, k1 = g.T0E[e]
        n0, n1 = g.E0E[e]
        g.markE0TE0T[(n0, n1)].append((k0, k1))
        g.markE0TE0T[(n1, n0)].append((k1, k0))
    return g


def map_to_physical(g, x1, x2):
    """F_k(x^) for all k at reference points (x1, x2): arrays [K, R] of x^1 and x^2 (eq. affinemappings)."""
    x1 = np.asarray(x1, dtype=np.float64)[None, :]
    x2 = np.asarray(x2, dtype=np.float64)[None, :]
    X = g.B[:, 0, 0:1] * x1 + g.B[:, 0, 1:2] * x2 + g.coordV0T[:, 0, 0:1]
    Y = g.B[:, 1, 0:1] * x1 + g.B[:, 1, 1:2] * x2 + g.coordV0T[:, 0, 1:2]
    return X, Y
