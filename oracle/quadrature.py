"""Quadrature rules on the reference triangle and on (0, 1) (Sec. 3.3, routines quadRule1D/2D).

Triangle rules (weights sum to |T^| = 1/2, points strictly inside T^):

* degree 1: centroid rule;
* degree 2: 3-point rule with points (1/6, 1/6), (2/3, 1/6), (1/6, 2/3);
* degree 3: the paper's 4-point rule is printed with 9 significant digits only and
  is exact to about 1e-10; a degree-3 request is served by the degree-4 rule;
* degree 4: 6-point rule (Strang-Fix / Cowper), two three-point orbits, constants
  to 15 digits as the paper prints them;
* degree 5: 7-point rule (Radon / Stroud) in closed form;
* degree 6: 12-point rule (Cowper), two three-point orbits and one six-point orbit,
  constants to 15 digits as the paper prints them;
* degree q >= 7: collapsed tensor Gauss rule (the paper calls a third-party routine
  here).  With x1 = u, x2 = (1 - u) v the Jacobian is (1 - u); u takes the n-point
  Gauss-Jacobi rule for the weight (1 - u) on (0, 1) and v the n-point Gauss-Legendre
  rule, n = ceil((q + 1) / 2).  Points are ordered u-major.

Edge rule: n-point Gauss-Legendre on (0, 1), sorted ascending, exact to degree 2n - 1.

Parity: pinned (exactness on all monomials up to the stated degree).
"""
from math import ceil, sqrt

import numpy as np
from scipy.special import roots_jacobi


def gauss_legendre_01(n):
    """n-point Gauss-Legendre rule on (0, 1): (points ascending, weights summing to 1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    order = np.argsort(x)
    return (x[order] + 1.0) / 2.0, w[order] / 2.0


def edge_points_for_degree(q):
    """Number of Gauss points for exactness of degree q on an edge."""
    return max(1, ceil((q + 1) / 2))


def _orbit3(a, w):
    """Three points with barycentric coordinates (a, a, 1 - 2a), each with weight w."""
    b = 1.0 - 2.0 * a
    return [(a, a, w), (b, a, w), (a, b, w)]


def _orbit6(a, b, w):
    """Six points with barycentric coordinates the permutations of (a, b, 1 - a - b)."""
    c = 1.0 - a - b
    return [(a, b, w), (b, a, w), (a, c, w), (c, a, w), (b, c, w), (c, b, w)]


def _collapsed(q):
    n = max(1, ceil((q + 1) / 2))
    # Gauss-Jacobi on (-1, 1) for weight (1 - t)^1 (1 + t)^0, mapped to u in (0, 1):
    # (1 - t) = 2 (1 - u), dt = 2 du  ->  weights scale by 1/4
    t, wt = roots_jacobi(n, 1.0, 0.0)
    u = (t + 1.0) / 2.0
    wu = wt / 4.0
    v, wv = gauss_legendre_01(n)
    pts = []
    for i in range(n):
        for j in range(n):
            pts.append((u[i], (1.0 - u[i]) * v[j], wu[i] * wv[j]))
    return pts


def triangle_rule(q):
    """Rule exact to degree >= q on T^: arrays (x1, x2, w)."""
    q = max(int(q), 1)
    if q == 1:
        pts = [(1.0 / 3.0, 1.0 / 3.0, 0.5)]
    elif q == 2:
        pts = [(1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0), (2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0),
               (1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0)]
    elif q in (3, 4):
        pts = _orbit3(0.445948490915965, 0.111690794839005) + \
              _orbit3(0.091576213509771, 0.054975871827661)
    elif q == 5:
        r15 = sqrt(15.0)
        a1, a2 = (6.0 - r15) / 21.0, (6.0 + r15) / 21.0
        w1, w2 = (155.0 - r15) / 2400.0, (155.0 + r15) / 2400.0
        pts = [(1.0 / 3.0, 1.0 / 3.0, 9.0 / 80.0)] + _orbit3(a1, w1) + _orbit3(a2, w2)
    elif q == 6:
        pts = _orbit3(0.063089014491502, 0.025422453185103) + \
              _orbit3(0.249286745170910, 0.058393137863189) + \
              _orbit6(0.053145049844816, 0.310352451033785, 0.041425537809187)
    else:
        pts = _collapsed(q)
    arr = np.array(pts, dtype=np.float64)
    return arr[:, 0].copy(), arr[:, 1].copy(), arr[:, 2].copy()


def gamma_map(n, s):
    """Parametrisation of reference edge n = 0, 1, 2 (the paper's E^_1..E^_3), eq. gammaMap."""
    s = np.asarray(s, dtype=np.float64)
    if n == 0:
        return 1.0 - s, s
    if n == 1:
        return np.zeros_like(s), 1.0 - s
    return s, np.zeros_like(s)


def theta_map(nm, np_, x1, x2):
    """Edge-to-edge map theta^_{n- n+} of eq. mapEE (0-based edge indices)."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    z = np.zeros_like(x1)
    table = {
        (0, 0): (1.0 - x1, 1.0 - x2), (0, 1): (z, x2), (0, 2): (x1, z),
        (1, 0): (1.0 - x2, x2), (1, 1): (z, 1.0 - x2), (1, 2): (x2, z),
        (2, 0): (x1, 1.0 - x1), (2, 1): (z, x1), (2, 2): (1.0 - x1, z),
    }
    return table[(nm, np_)]
