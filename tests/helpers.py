"""Shared helpers of the GPU tests: matched oracle / CUDA problems on the same seeded inputs."""
import numpy as np

import workloads as W

MIXES = {"dirichlet": ((1, 2, 3, 4), ()), "neumann": ((), (1, 2, 3, 4)), "mixed": ((2, 4), (1, 3))}


def mesh(n, mix="mixed", jitter=0.2, seed=1):
    cV, V0T, side = W.square_mesh(n, jitter=jitter, seed=seed)
    dr, nr = MIXES[mix]
    return cV, V0T, W.boundary_types(side, dr, nr)


def smooth_d(x, y):
    return 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.3 * x * y


def gpu_solver(cV, V0T, bdr, p, quad_order=0):
    from paper_1408_3877_gb300 import festung as F
    return F.Solver(cV, V0T, bdr).setup(p, quad_order)


def samples(solver, func):
    xy, _ = solver.quad_points()
    return func(xy[..., 0], xy[..., 1])


def edge_samples(solver, func):
    _, exy = solver.quad_points()
    return func(exy[..., 0], exy[..., 1])


def rounding_bound(S_abs, x, eps):
    """A bound on the rounding error of y = S x: eps * |S| |x| summed in 2-norm."""
    return eps * np.linalg.norm(S_abs @ np.abs(x))


def factored_scale(L, D, tau, x):
    """Rounding scale of y = S x evaluated in factors, as the kernels do (Z^m = -M^{-1}
    B_m x first, then M x + tau (eta S_t x + sum_m A_m Z^m)): the same product with every
    factor and x replaced by its absolute value.  It bounds the magnitude of every partial
    sum of the evaluation, which |S| |x| (after the cancellations inside S) does not."""
    ax = np.abs(np.asarray(x).ravel())
    A = L.Am(D)
    minv = abs(L.Minv)
    flux = sum(abs(A[m]) @ (minv @ (abs(L.Bm[m]) @ ax)) for m in range(2))
    return abs(L.M) @ ax + tau * (L.eta * (abs(L.St) @ ax) + flux)


def to_gpu_layout(x, K, N, dtype, order):
    """Caller-order K x N coefficients -> device layout N x K in the library's internal order."""
    import torch
    xi = np.asarray(x).reshape(K, N)[np.asarray(order)]
    return torch.tensor(np.ascontiguousarray(xi.T), dtype=dtype, device="cuda")


def from_gpu_layout(y, order):
    """Device layout N x K (internal order) -> caller-order K x N."""
    yi = y.double().cpu().numpy().T
    out = np.empty_like(yi)
    out[np.asarray(order)] = yi
    return out


def patch_oracle_rows(cV, V0T, bdr, p, dfun, x, tau, ks, quad_order=None, eta=1.0):
    """Rows k of S x (and of its factored rounding scale, see factored_scale) computed by
    the oracle on the 2-ring patch of each k.

    y_k depends on x and d in the 2-ring of k only (the flux unknowns of k and of its
    neighbours).  Edges that leave the patch get an arbitrary boundary type; they touch
    only flux unknowns of 2-ring elements, which y_k does not use.
    """
    from oracle.solve import LDG
    V0T = np.asarray(V0T)
    K = V0T.shape[0]
    N = (p + 1) * (p + 2) // 2
    xk = np.asarray(x).reshape(K, N)
    # triangle adjacency through shared vertex pairs (vectorised)
    va = V0T[:, [1, 2, 0]].ravel().astype(np.int64)
    vb = V0T[:, [2, 0, 1]].ravel().astype(np.int64)
    key = np.minimum(va, vb) * (int(V0T.max()) + 1) + np.maximum(va, vb)
    order = np.argsort(key, kind="stable")
    ks_sorted = key[order]
    same = np.nonzero(ks_sorted[1:] == ks_sorted[:-1])[0]
    h0, h1 = order[same], order[same + 1]
    nbr = -np.ones(3 * K, dtype=np.int64)
    nbr[h0] = h1 // 3
    nbr[h1] = h0 // 3
    nbr = nbr.reshape(K, 3)

    out, scale = [], []
    for k in ks:
        ring = {k}
        for _ in range(2):
            ring |= {int(j) for i in ring for j in nbr[i] if j >= 0}
        ring = sorted(ring)
        loc = {g: i for i, g in enumerate(ring)}
        T = V0T[ring]
        verts, inv = np.unique(T.ravel(), return_inverse=True)
        T2 = inv.reshape(T.shape)
        b2 = np.array(bdr)[ring].copy()
        for i, g in enumerate(ring):
            for n in range(3):
                if nbr[g, n] >= 0 and int(nbr[g, n]) not in loc:
                    b2[i, n] = 2
        L = LDG(np.asarray(cV)[verts], T2, b2, p, quad_order=quad_order, eta=eta)
        D = L.project(dfun)
        S = L.operator(D, tau)
        xr = xk[ring].ravel()
        y = (S @ xr).reshape(len(ring), N)
        sc = factored_scale(L, D, tau, xr).reshape(len(ring), N)
        out.append(y[loc[k]])
        scale.append(sc[loc[k]])
    return np.array(out), np.array(scale)


def patch_case(p):
    """A stationary problem whose exact solution lies in the discrete space (LDG is
    consistent, so the discrete solution is the projection of c): for p = 1, c linear;
    for p >= 2, c quadratic (z = -grad c is then linear).  d is constant, f = -d lap c.
    Returns c, d, f and g_N = -grad c . nu on the sides of the unit square (outward
    normals (0, -1) on y = 0, (1, 0) on x = 1, (0, 1) on y = 1, (-1, 0) on x = 0)."""
    d0 = 2.5
    if p == 1:
        def c(x, y):
            return 1.0 + 2.0 * x - 3.0 * y

        def grad(x, y):
            return 2.0 + 0.0 * x, -3.0 + 0.0 * y
        lap = 0.0
    else:
        def c(x, y):
            return 1.0 + 2.0 * x - 3.0 * y + 0.5 * x * x - x * y + 0.25 * y * y

        def grad(x, y):
            return 2.0 + x - y, -3.0 - x + 0.5 * y
        lap = 1.5

    def d(x, y):
        return d0 + 0.0 * x

    def f(x, y):
        return -d0 * lap + 0.0 * x

    def gN(x, y):
        cx, cy = grad(x, y)
        eps = 1e-12
        return np.where(np.abs(y) < eps, cy, np.where(np.abs(y - 1) < eps, -cy,
                                                      np.where(np.abs(x) < eps, cx, -cx)))
    return c, d, f, gN
