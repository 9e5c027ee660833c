"""Pins of the oracle's grid lists and L2 projection."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import basis, grid, project

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _jittered(n=6, seed=3):
    cV, V0T, side = W.square_mesh(n, jitter=0.2, seed=seed)
    return cV, V0T, W.boundary_types(side, dirichlet=(2, 4), neumann=(1, 3))


def test_grid_identities():
    cV, V0T, bdr = _jittered()
    g = grid.generate_grid_data(cV, V0T, bdr)
    K = g.numT
    # closed triangle: sum_n |E_kn| nu_kn = 0
    s = np.einsum("kn,knm->km", g.areaE0T, g.nuE0T)
    np.testing.assert_allclose(s, 0.0, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(g.nuE0T, axis=-1), 1.0, atol=1e-15)
    # exterior normals: point away from the centroid
    cen = g.coordV0T.mean(axis=1)
    mid = 0.5 * (g.coordV0T[:, [1, 2, 0]] + g.coordV0T[:, [2, 0, 1]])
    assert np.all(np.einsum("knm,knm->kn", mid - cen[:, None], g.nuE0T) > 0)
    # 2 |T| = det B and the areas tile the unit square
    np.testing.assert_allclose(g.areaT.sum(), 1.0, atol=1e-14)
    nint = np.sum(g.T0E[:, 1] >= 0)
    nb = g.numE - nint
    assert 3 * K == 2 * nint + nb
    for e in range(g.numE):
        for sl in range(2):
            k = g.T0E[e, sl]
            if k >= 0:
                assert g.E0T[k, g.E0E[e, sl]] == e
    # neighbours across an interior edge see opposite normals and equal lengths
    for (nm, npl), pairs in g.markE0TE0T.items():
        for km, kp in pairs:
            np.testing.assert_allclose(g.nuE0T[km, nm], -g.nuE0T[kp, npl], atol=1e-15)
            assert abs(g.areaE0T[km, nm] - g.areaE0T[kp, npl]) < 1e-15


def test_two_triangle_grid_of_visualization_example():
    # Sec. 3.10: vertices (0,-1), (sqrt3,0), (0,1), (-sqrt3,0); triangles (4,1,3), (1,2,3)
    r3 = np.sqrt(3.0)
    cV = np.array([[0.0, -1.0], [r3, 0.0], [0.0, 1.0], [-r3, 0.0]])
    V0T = np.array([[3, 0, 2], [0, 1, 2]])
    bdr = np.array([[0, 1, 1], [1, 0, 1]])  # the shared edge (0,-1)-(0,1) is interior
    g = grid.generate_grid_data(cV, V0T, bdr)
    assert g.numE == 5
    np.testing.assert_allclose(g.areaT, [r3, r3])
    assert g.markE0TE0T[(0, 1)] == [(0, 1)] and g.markE0TE0T[(1, 0)] == [(1, 0)]


def test_invalid_meshes_rejected():
    cV, V0T, bdr = _jittered(3)
    with pytest.raises(ValueError):
        grid.generate_grid_data(cV, V0T[:, ::-1], bdr)          # clockwise
    bad = bdr.copy()
    bad[bad > 0] = 0
    with pytest.raises(ValueError):
        grid.generate_grid_data(cV, V0T, bad)                    # boundary edge without type


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_projection_reproduces_polynomials(p):
    cV, V0T, bdr = _jittered(4)
    g = grid.generate_grid_data(cV, V0T, bdr)
    N = basis.num_dofs(p)
    rng = np.random.default_rng(p)
    coef = rng.standard_normal((p + 1, p + 1))

    def poly(x, y):
        return sum(coef[a, b] * x**a * y**b for a in range(p + 1) for b in range(p + 1 - a))

    C = project.project(g, poly, N, 2 * p)
    x1, x2 = np.array([0.2, 0.5, 0.1]), np.array([0.3, 0.1, 0.7])
    X, Y = grid.map_to_physical(g, x1, x2)
    np.testing.assert_allclose(project.evaluate(C, x1, x2), poly(X, Y), atol=1e-11)


def test_two_triangle_projection_ranges():
    r3 = np.sqrt(3.0)
    cV = np.array([[0.0, -1.0], [r3, 0.0], [0.0, 1.0], [-r3, 0.0]])
    V0T = np.array([[3, 0, 2], [0, 1, 2]])
    bdr = np.array([[0, 1, 1], [1, 0, 1]])
    g = grid.generate_grid_data(cV, V0T, bdr)

    def f(x, y):
        return np.where(x < 0, x**2 - y**2 - 1, -x**2 - y**2 + 1)

    nodes = {1: ([1 / 3], [1 / 3]), 3: ([0, 1, 0], [0, 0, 1]),
             6: ([0, 1, 0, 0.5, 0, 0.5], [0, 0, 1, 0.5, 0.5, 0])}
    gold = np.loadtxt(os.path.join(GOLDEN, "two_triangle_ranges.txt"))
    for N, lo, hi in gold:
        N = int(N)
        p = {1: 0, 3: 1, 6: 2}[N]
        C = project.project(g, f, N, p + 2)
        vals = project.evaluate(C, np.array(nodes[N][0], float), np.array(nodes[N][1], float))
        assert abs(vals.min() - lo) < 1e-12 and abs(vals.max() - hi) < 1e-12, (N, vals.min(), vals.max())


@pytest.mark.parametrize("p", [0, 2, 4])
def test_l2_error_absolute_scale_closed_forms(p):
    """Absolute scale of the L2 error (Sec. 3.5), which convergence rates cannot see:
    on the unit square (jittered and regular meshes) ||0 - 1|| = 1, ||0 - x|| = 1/sqrt(3),
    ||0 - xy|| = 1/3, and with c_h the projection of 1, ||c_h - (1 + x)|| = 1/sqrt(3).
    A dropped factor 2, a missing |T_k| weight or a mis-evaluated c_h changes these."""
    from oracle import quadrature
    for jitter in (0.0, 0.25):
        cV, V0T, side = W.square_mesh(5, jitter=jitter, seed=7)
        bdr = W.boundary_types(side, dirichlet=(1, 2, 3, 4))
        g = grid.generate_grid_data(cV, V0T, bdr)
        N = basis.num_dofs(p)
        Z = np.zeros((g.numT, N))
        qT = max(4, 2 * p + 2)  # exact for the degree-4 integrand (xy)^2
        assert project.l2_error(g, Z, lambda x, y: 1.0 + 0.0 * x, qT) == pytest.approx(1.0, rel=1e-13)
        assert project.l2_error(g, Z, lambda x, y: x, qT) == pytest.approx(1.0 / np.sqrt(3.0), rel=1e-13)
        assert project.l2_error(g, Z, lambda x, y: x * y, qT) == pytest.approx(1.0 / 3.0, rel=1e-13)
        one = project.project(g, lambda x, y: 1.0 + 0.0 * x, N, max(1, 2 * p))
        assert project.l2_error(g, one, lambda x, y: 1.0 + x, qT) == pytest.approx(1.0 / np.sqrt(3.0), rel=1e-13)
        # a sliver of the domain: the error of c_h = 0 against the indicator-like data
        # 1 on one triangle only is sqrt(|T_k|)
        k = 3
        mask = np.zeros(g.numT)
        mask[k] = 1.0
        q1, q2, _ = quadrature.triangle_rule(qT)
        X, _ = grid.map_to_physical(g, q1, q2)
        ind = np.broadcast_to(mask[:, None], X.shape)
        err = project.l2_error(g, Z, lambda x, y: ind, qT)
        assert err == pytest.approx(np.sqrt(g.areaT[k]), rel=1e-13)
