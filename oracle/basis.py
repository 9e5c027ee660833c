"""Orthonormal modal basis on the reference triangle (Sec. 2.4.1, routines phi/gradPhi).

The paper gives N = (p+1)(p+2)/2 functions per order p <= 4 on the unit reference
triangle T^ = {x1 >= 0, x2 >= 0, x1 + x2 <= 1}, orthonormal in L2(T^) (Sec. 2.4.1).
Their closed forms for p <= 2 are printed in Sec. 2.4.1.

Here the same 15 functions are obtained by exact Gram-Schmidt orthogonalisation of
the monomials, taken degree by degree in the order

    1 | x1, x2 | x1^2, x2^2, x1 x2 | x1^3, x1^2 x2, x1 x2^2, x2^3 |
    x1^4, x1^3 x2, x1^2 x2^2, x1 x2^3, x2^4

in rational arithmetic, with the exact reference-triangle moments
    int_T^ x1^a x2^b = a! b! / (a + b + 2)!,
then normalised in FP64.  Gram-Schmidt fixes each function up to its sign; the sign
is chosen so that the value at the vertex a^_1 = (0, 0) has the sign the paper's
functions have there (``_SIGN_AT_ORIGIN``).  The result coincides with the paper's
phi_1..phi_15; tests pin it against the p <= 2 closed forms printed in Sec. 2.4.1
and against exact orthonormality.

Parity: pinned (closed forms for p <= 2, exact orthonormality, finite differences
for the gradients).
"""
from fractions import Fraction
from math import factorial, sqrt

import numpy as np

# monomial exponents (a, b) for x1^a x2^b, in the Gram-Schmidt order described above
MONOMIALS = [
    (0, 0),
    (1, 0), (0, 1),
    (2, 0), (0, 2), (1, 1),
    (3, 0), (2, 1), (1, 2), (0, 3),
    (4, 0), (3, 1), (2, 2), (1, 3), (0, 4),
]
# sign of phi_i(0, 0) for the paper's basis, i = 1..15
_SIGN_AT_ORIGIN = [+1, +1, +1, +1, -1, +1, -1, -1, -1, -1, +1, +1, +1, +1, +1]

PMAX = 4


def num_dofs(p):
    """N = (p+1)(p+2)/2 local degrees of freedom (Sec. 2.4.1)."""
    return (p + 1) * (p + 2) // 2


def _moment(a, b):
    """Exact int over T^ of x1^a x2^b."""
    return Fraction(factorial(a) * factorial(b), factorial(a + b + 2))


def _inner(f, g):
    """Exact L2(T^) inner product of polynomials given as {(a, b): Fraction}."""
    s = Fraction(0)
    for (a, b), c in f.items():
        for (d, e), k in g.items():
            s += c * k * _moment(a + d, b + e)
    return s


def _gram_schmidt():
    """Exact orthogonal (not yet normalised) polynomials and their squared norms."""
    polys, norms = [], []
    for mon in MONOMIALS:
        f = {mon: Fraction(1)}
        for q, nq in zip(polys, norms):
            c = _inner({mon: Fraction(1)}, q) / nq
            for key, val in q.items():
                f[key] = f.get(key, Fraction(0)) - c * val
        f = {k: v for k, v in f.items() if v != 0}
        polys.append(f)
        norms.append(_inner(f, f))
    return polys, norms


def _build_coefficients():
    polys, norms = _gram_schmidt()
    coef = np.zeros((len(MONOMIALS), len(MONOMIALS)))  # coef[i, monomial index]
    for i, (f, nf) in enumerate(zip(polys, norms)):
        scale = 1.0 / sqrt(float(nf))
        val0 = f.get((0, 0), Fraction(0))
        s = 1.0 if val0 == 0 else (1.0 if val0 > 0 else -1.0)
        scale *= s * _SIGN_AT_ORIGIN[i]
        for m, mon in enumerate(MONOMIALS):
            if mon in f:
                coef[i, m] = float(f[mon]) * scale
    return coef, polys, norms


COEF, _EXACT_POLYS, _EXACT_NORMS = _build_coefficients()


def exact_gram_matrix(N):
    """Exact Gram matrix of the first N orthogonal polynomials (diagonal by construction)."""
    return [[_inner(_EXACT_POLYS[i], _EXACT_POLYS[j]) for j in range(N)] for i in range(N)]


def phi(i, x1, x2):
    """phi^_i at points (x1, x2) of T^, i = 0..14 (0-based; the paper counts 1..15)."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    out = np.zeros(np.broadcast(x1, x2).shape)
    for m, (a, b) in enumerate(MONOMIALS):
        c = COEF[i, m]
        if c != 0.0:
            out = out + c * x1**a * x2**b
    return out


def grad_phi(i, m, x1, x2):
    """Component m (0: d/dx1^, 1: d/dx2^) of the gradient of phi^_i at (x1, x2)."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    out = np.zeros(np.broadcast(x1, x2).shape)
    for k, (a, b) in enumerate(MONOMIALS):
        c = COEF[i, k]
        if c == 0.0:
            continue
        if m == 0 and a > 0:
            out = out + c * a * x1 ** (a - 1) * x2**b
        elif m == 1 and b > 0:
            out = out + c * b * x1**a * x2 ** (b - 1)
    return out


def phi_table(N, x1, x2):
    """Matrix [len(x1), N] of phi^_j(x_r)."""
    return np.stack([phi(j, x1, x2) for j in range(N)], axis=-1)


def grad_phi_table(N, x1, x2):
    """Array [len(x1), N, 2] of grad phi^_j(x_r)."""
    return np.stack(
        [np.stack([grad_phi(j, m, x1, x2) for m in range(2)], axis=-1) for j in range(N)],
        axis=-2,
    )
