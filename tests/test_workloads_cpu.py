"""The seeded input generators (no method arithmetic): the Gaussian-field gradient used to
manufacture sources for d = exp(g), and the specs of the batched workload."""
import numpy as np

import workloads as W


def test_grf_gradient_is_the_interpolant_derivative():
    f = W.GaussianField(3, 0.1)
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 1, 500), rng.uniform(0, 1, 500)
    g, gx, gy = W.grf_gradient(f, x, y)
    assert np.array_equal(g, f(x, y))
    h = 1e-7  # central differences inside a cell of the bilinear interpolant
    assert np.max(np.abs(gx - (f(x + h, y) - f(x - h, y)) / (2 * h))) < 1e-5
    assert np.max(np.abs(gy - (f(x, y + h) - f(x, y - h)) / (2 * h))) < 1e-5


def test_grf_coefficient_and_manufactured_source():
    field = W.GaussianField(7, 0.05)
    dfun = W.grf_coefficient(field)
    man = W.Manufactured(dfun)
    x, y = np.array([0.31, 0.77]), np.array([0.52, 0.18])
    d, dx, dy = dfun(0.0, x, y)
    assert np.allclose(d, np.exp(field(x, y)))
    # f(t) = exp(-t) f(0) for the manufactured c and a time-independent d
    assert np.allclose(man.f(0.3, x, y), np.exp(-0.3) * man.f(0.0, x, y))


def test_batched_specs():
    specs = W.batched_problems(512, 2024)
    assert len(specs) == 512
    assert all(16 <= s["n"] <= 192 and s["p"] in (1, 2, 3) and 0.02 <= s["length"] <= 0.2 for s in specs)
    assert specs == W.batched_problems(512, 2024)  # seeded
    K = sum(2 * s["n"] ** 2 for s in specs)
    assert 1.0e7 < K < 1.8e7  # ~1.4e7 triangles
