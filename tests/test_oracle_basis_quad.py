"""Pins of the oracle's basis and quadrature against what the paper and mathematics fix."""
from math import factorial

import numpy as np
import pytest

from oracle import basis, quadrature

SQ2, SQ3, SQ5, SQ6 = np.sqrt(2.0), np.sqrt(3.0), np.sqrt(5.0), np.sqrt(6.0)

# closed forms for p <= 2 as printed in Sec. 2.4.1 (local basis representation)
PRINTED_P2 = [
    lambda x, y: SQ2 + 0.0 * x,
    lambda x, y: 2.0 - 6.0 * x,
    lambda x, y: 2.0 * SQ3 * (1.0 - x - 2.0 * y),
    lambda x, y: SQ6 * ((10.0 * x - 8.0) * x + 1.0),
    lambda x, y: SQ3 * ((5.0 * x - 4.0) * x + (-15.0 * y + 12.0) * y - 1.0),
    lambda x, y: 3.0 * SQ5 * ((3.0 * x + 8.0 * y - 4.0) * x + (3.0 * y - 4.0) * y + 1.0),
]


def _points(n=64, seed=0):
    r = np.random.default_rng(seed)
    x = r.random(n)
    y = r.random(n) * (1.0 - x)
    return x, y


def exact_moment(a, b):
    return factorial(a) * factorial(b) / factorial(a + b + 2)


def test_basis_matches_printed_closed_forms():
    x, y = _points()
    for i, f in enumerate(PRINTED_P2):
        np.testing.assert_allclose(basis.phi(i, x, y), f(x, y), rtol=0, atol=1e-13)


def test_basis_orthonormal_exact_moments():
    # M^ = I (Sec. 2.4.1, eq. hatM) with exact monomial integration, all 15 functions
    C = basis.COEF
    mom = np.array([[exact_moment(a + c, b + d) for (c, d) in basis.MONOMIALS]
                    for (a, b) in basis.MONOMIALS])
    G = C @ mom @ C.T
    # monomial coefficients reach ~1e4, so this FP64 evaluation carries ~1e-12 of rounding
    np.testing.assert_allclose(G, np.eye(15), atol=2e-11)


def test_basis_orthonormal_by_high_order_quadrature():
    x1, x2, w = quadrature.triangle_rule(10)
    P = basis.phi_table(15, x1, x2)
    np.testing.assert_allclose(P.T @ (w[:, None] * P), np.eye(15), atol=1e-12)


def test_basis_degree_structure():
    # phi_i has exactly the degree of its slot: N(p-1) < i <= N(p) <=> degree p
    for i, (a, b) in enumerate(basis.MONOMIALS):
        deg = a + b
        nz = [basis.MONOMIALS[m] for m in range(15) if abs(basis.COEF[i, m]) > 1e-12]
        assert max(sum(t) for t in nz) == deg


def test_gradient_matches_finite_differences():
    x, y = _points(32, seed=1)
    x = 0.05 + 0.9 * x * 0.9
    y = 0.05 + y * 0.8 * (0.95 - x)
    h = 1e-6
    for i in range(15):
        fd1 = (basis.phi(i, x + h, y) - basis.phi(i, x - h, y)) / (2 * h)
        fd2 = (basis.phi(i, x, y + h) - basis.phi(i, x, y - h)) / (2 * h)
        np.testing.assert_allclose(basis.grad_phi(i, 0, x, y), fd1, atol=2e-6 * (1 + np.abs(fd1).max()))
        np.testing.assert_allclose(basis.grad_phi(i, 1, x, y), fd2, atol=2e-6 * (1 + np.abs(fd2).max()))


@pytest.mark.parametrize("q", list(range(1, 13)))
def test_triangle_rule_exactness(q):
    x1, x2, w = quadrature.triangle_rule(q)
    assert np.all(w > 0)
    assert np.all(x1 > 0) and np.all(x2 > 0) and np.all(x1 + x2 < 1)
    eff = 4 if q == 3 else q
    for a in range(eff + 1):
        for b in range(eff + 1 - a):
            ex = exact_moment(a, b)
            got = np.sum(w * x1**a * x2**b)
            assert abs(got - ex) <= 5e-15 * max(1.0, 1.0 / ex) * ex + 1e-16, (q, a, b, got, ex)


def test_collapsed_rule_sizes():
    # degree 8 (p = 4) -> 5 x 5 points; degree 7 -> 4 x 4
    assert quadrature.triangle_rule(8)[0].size == 25
    assert quadrature.triangle_rule(7)[0].size == 16


@pytest.mark.parametrize("n", list(range(1, 10)))
def test_gauss_legendre(n):
    s, w = quadrature.gauss_legendre_01(n)
    assert np.all(np.diff(s) > 0)
    np.testing.assert_allclose(s + s[::-1], 1.0, atol=1e-15)
    np.testing.assert_allclose(w, w[::-1], atol=1e-15)
    for k in range(2 * n):
        assert abs(np.sum(w * s**k) - 1.0 / (k + 1)) < 1e-15


def test_theta_maps_reverse_orientation():
    # Sec. 3.6.4: every edge-to-edge map reverses the edge orientation,
    # theta_{n- n+}(gamma_{n-}(s)) = gamma_{n+}(1 - s)
    s = np.linspace(0.0, 1.0, 11)
    for nm in range(3):
        x1, x2 = quadrature.gamma_map(nm, s)
        for npl in range(3):
            y1, y2 = quadrature.theta_map(nm, npl, x1, x2)
            z1, z2 = quadrature.gamma_map(npl, 1.0 - s)
            np.testing.assert_allclose(y1, z1, atol=1e-15)
            np.testing.assert_allclose(y2, z2, atol=1e-15)


def test_gamma_maps_are_the_edges_opposite_the_vertices():
    # edge n of T^ lies opposite vertex n and runs counter-clockwise (Fig. reference triangle)
    verts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    for n in range(3):
        x1, x2 = quadrature.gamma_map(n, np.array([0.0, 1.0]))
        np.testing.assert_allclose([x1[0], x2[0]], verts[(n + 1) % 3])
        np.testing.assert_allclose([x1[1], x2[1]], verts[(n + 2) % 3])
