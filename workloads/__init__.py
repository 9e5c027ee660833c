"""Seeded synthetic inputs shared by the oracle, the tests, the smoke run and the bench.

This module only produces inputs: meshes of the unit square, boundary markers,
coefficient and data functions, random fields and random initial states.  It holds
none of the LDG method's arithmetic (no basis, quadrature, assembly or solve).

Mesh: the Friedrichs-Keller triangulation of the unit square used by the paper's
routine domainSquare (Sec. 4): vertex (ix h, iy h) has index iy + ix (n + 1); each
square is split along its (x + h, y)-(x, y + h) diagonal into the counter-clockwise
triangles {(x, y), (x + h, y), (x, y + h)} and {(x + h, y), (x + h, y + h), (x, y + h)};
all lower-left triangles come first, then all upper-right ones, both in the vertex
order.  Boundary ids: 1 south (y = 0), 2 east (x = 1), 3 north (y = 1), 4 west (x = 0).
Optional jitter moves every interior vertex coordinate by an independent seeded
U(-a h, +a h).

Local edge n of a triangle lies opposite its vertex n.  Boundary types per local
edge: 0 interior, 1 Dirichlet, 2 Neumann.
"""
import numpy as np

INTERIOR, DIRICHLET, NEUMANN = 0, 1, 2


def square_mesh(n, jitter=0.0, seed=0):
    """(coordV [numV, 2], V0T [K, 3] int32, side [K, 3] int8 boundary id or 0)."""
    n = int(n)
    h = 1.0 / n
    ix, iy = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    ixf, iyf = ix.ravel(), iy.ravel()                      # vertex v = iy + ix (n + 1)
    coordV = np.stack([ixf * h, iyf * h], axis=1).astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        inner = (ixf > 0) & (ixf < n) & (iyf > 0) & (iyf < n)
        d = rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 2))
        coordV[inner] += d
    sq_ix, sq_iy = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    o = (sq_iy + sq_ix * (n + 1)).ravel()
    V0T1 = np.stack([o, o + n + 1, o + 1], axis=1)
    V0T2 = np.stack([o + n + 1, o + n + 2, o + 1], axis=1)
    V0T = np.concatenate([V0T1, V0T2]).astype(np.int32)
    # boundary id of each local edge (edge n joins vertices n+1 and n+2)
    va = V0T[:, [1, 2, 0]]
    vb = V0T[:, [2, 0, 1]]
    xa, ya = ixf[va], iyf[va]
    xb, yb = ixf[vb], iyf[vb]
    side = np.zeros(V0T.shape, dtype=np.int8)
    side[(ya == 0) & (yb == 0)] = 1
    side[(xa == n) & (xb == n)] = 2
    side[(ya == n) & (yb == n)] = 3
    side[(xa == 0) & (xb == 0)] = 4
    return coordV, V0T, side


def boundary_types(side, dirichlet=(), neumann=()):
    bdr = np.zeros(side.shape, dtype=np.int8)
    for i in dirichlet:
        bdr[side == i] = DIRICHLET
    for i in neumann:
        bdr[side == i] = NEUMANN
    if np.any((side > 0) & (bdr == 0)):
        raise ValueError("every boundary id needs a type")
    return bdr


# ---------------------------------------------------------------------------
# manufactured solution c = cos(7x) cos(7y) exp(-t) and its data
# ---------------------------------------------------------------------------
class Manufactured:
    """c, d, f = dt c - div(d grad c), c_D = c and g_N = -grad c . nu on the unit square.

    ``d`` and its gradient are given as callables d(t, x, y) -> (d, d_x, d_y).
    """

    def __init__(self, dfun, stationary=False):
        self.dfun = dfun
        self.stationary = stationary

    def _tf(self, t):
        return 1.0 if self.stationary else np.exp(-t)

    def c(self, t, x, y):
        return np.cos(7 * x) * np.cos(7 * y) * self._tf(t)

    def cx(self, t, x, y):
        return -7 * np.sin(7 * x) * np.cos(7 * y) * self._tf(t)

    def cy(self, t, x, y):
        return -7 * np.cos(7 * x) * np.sin(7 * y) * self._tf(t)

    def d(self, t, x, y):
        return self.dfun(t, x, y)[0]

    def f(self, t, x, y):
        d, dx, dy = self.dfun(t, x, y)
        c = self.c(t, x, y)
        lap = -98.0 * c
        dtc = 0.0 if self.stationary else -c
        return dtc - (dx * self.cx(t, x, y) + dy * self.cy(t, x, y) + d * lap)

    def gN(self, t, x, y):
        """-grad c . nu with nu the exterior normal of the nearest side of the square."""
        dist = np.stack([np.abs(y), np.abs(1 - x), np.abs(1 - y), np.abs(x)])
        s = np.argmin(dist, axis=0)
        cx, cy = self.cx(t, x, y), self.cy(t, x, y)
        return np.choose(s, [cy, -cx, -cy, cx])


def d_config1(t, x, y):
    s = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    d = 1.0 + 0.5 * s
    dx = 0.5 * 2 * np.pi * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    dy = 0.5 * 2 * np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    return d, dx, dy


def d_config2(t, x, y):
    a = 0.5 * (1.0 + t)
    d = 1.0 + a * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    dx = a * 2 * np.pi * np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y)
    dy = -a * 2 * np.pi * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    return d, dx, dy


def d_verification(t, x, y):
    """d = exp(x + y) of the verification problem (Sec. 3.9)."""
    e = np.exp(x + y)
    return e, e, e


# ---------------------------------------------------------------------------
# Gaussian random field with squared-exponential covariance
# ---------------------------------------------------------------------------
class GaussianField:
    """Seeded stationary Gaussian field g with covariance var * exp(-r^2 / (2 l^2)).

    Spectral synthesis on a periodic grid covering [-pad, 1 + pad]^2 with spacing
    <= l / 8, evaluated by bilinear interpolation.  The grid variance is exactly
    ``variance``.
    """

    def __init__(self, seed, length, variance=1.0):
        self.length, self.variance = float(length), float(variance)
        pad = 3.0 * self.length
        span = 1.0 + 2.0 * pad
        m = int(2 ** np.ceil(np.log2(span / (self.length / 8.0))))
        m = max(m, 64)
        self.m, self.lo, self.dx = m, -pad, span / m
        rng = np.random.default_rng(seed)
        k = 2 * np.pi * np.fft.fftfreq(m, d=self.dx)
        kx, ky = np.meshgrid(k, k, indexing="ij")
        spec = np.exp(-0.5 * self.length**2 * (kx**2 + ky**2))
        amp = np.sqrt(spec / spec.sum() * self.variance)
        w = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        self.grid = np.real(np.fft.fft2(amp * w))

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        u = (x - self.lo) / self.dx
        v = (y - self.lo) / self.dx
        i = np.clip(np.floor(u).astype(np.int64), 0, self.m - 2)
        j = np.clip(np.floor(v).astype(np.int64), 0, self.m - 2)
        a, b = u - i, v - j
        G = self.grid
        return ((1 - a) * (1 - b) * G[i, j] + a * (1 - b) * G[i + 1, j]
                + (1 - a) * b * G[i, j + 1] + a * b * G[i + 1, j + 1])


def grf_gradient(field, x, y):
    """(g, g_x, g_y) of the bilinear interpolant of a GaussianField (its derivative
    inside each grid cell)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    u = (x - field.lo) / field.dx
    v = (y - field.lo) / field.dx
    i = np.clip(np.floor(u).astype(np.int64), 0, field.m - 2)
    j = np.clip(np.floor(v).astype(np.int64), 0, field.m - 2)
    a, b = u - i, v - j
    G = field.grid
    g00, g10, g01, g11 = G[i, j], G[i + 1, j], G[i, j + 1], G[i + 1, j + 1]
    g = (1 - a) * (1 - b) * g00 + a * (1 - b) * g10 + (1 - a) * b * g01 + a * b * g11
    gx = ((1 - b) * (g10 - g00) + b * (g11 - g01)) / field.dx
    gy = ((1 - a) * (g01 - g00) + a * (g11 - g10)) / field.dx
    return g, gx, gy


def grf_coefficient(field):
    """d = exp(g) with its gradient, as the callable d(t, x, y) -> (d, d_x, d_y) that
    Manufactured takes (time-independent)."""
    def d(t, x, y):
        g, gx, gy = grf_gradient(field, x, y)
        e = np.exp(g)
        return e, e * gx, e * gy
    return d


def batched_problems(nprob, seed):
    """Specs of the batched workload: per problem an n x n grid, n ~ U{16..192}, order
    p ~ U{1, 2, 3}, and its own Gaussian field length l ~ U[0.02, 0.2] (variance 1)."""
    rng = np.random.default_rng(seed)
    return [dict(n=int(rng.integers(16, 193)), p=int(rng.integers(1, 4)), length=float(rng.uniform(0.02, 0.2)),
                 grf_seed=int(rng.integers(0, 2**31 - 1))) for _ in range(nprob)]


def random_state(K, N, seed):
    """C0[k, j] ~ N(0, 1) / (1 + j): seeded normal coefficients scaled by basis index."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((K, N)) / (1.0 + np.arange(N))[None, :]


# ---------------------------------------------------------------------------
# the five workloads (shapes of the paper's test problems, Sec. 3.9 / 4 main script)
# ---------------------------------------------------------------------------
CONFIGS = {
    "square8_p1": dict(n=8, jitter=0.0, p=1, quad_order=3, dt=0.01, steps=10,
                        dirichlet=(1, 2, 3, 4), neumann=(), coeff="manufactured1"),
    "jitter256_p4": dict(n=256, jitter=0.2, p=4, quad_order=None, dt=1e-3, steps=100,
                          dirichlet=(2, 4), neumann=(1, 3), coeff="manufactured2", tol=1e-10),
    "grf1024_p2": dict(n=1024, jitter=0.0, p=2, quad_order=None, dt=1e-4, steps=50,
                        dirichlet=(), neumann=(1, 2, 3, 4), coeff="grf", grf_length=0.05),
    "grf128_p3": dict(n=128, jitter=0.2, p=3, quad_order=None, dt=1e-3, steps=20,
                       dirichlet=(), neumann=(1, 2, 3, 4), coeff="grf", grf_length=0.05),
    # 512 independent problems (specs from batched_problems), each with d = exp(g) of its own
    # field, the manufactured c and f of square8_p1, Dirichlet data from c on the whole boundary
    "batched512": dict(nprob=512, seed=2024, dt=1e-3, steps=20, tol=1e-10,
                        dirichlet=(1, 2, 3, 4), neumann=(), coeff="grf-manufactured"),
}
