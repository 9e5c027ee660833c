"""Why the inner operator of the mixed step stays FP32 and does not use BF16 tables.

Iterative refinement x += S~^{-1} (b - S x) converges only if the inner operator S~
is close enough to S relative to its conditioning.  The most favourable model of an
apply with BF16 tables is the assembled S (the oracle's CSR operator of the eliminated
step, Sec. 2.5 with z eliminated) with every entry rounded to BF16; a real BF16-table
apply also rounds the operands inside its contractions and errs more.  On a 32 x 32
jittered mesh at p = 4 and the time step of the 256 x 256 workload (tau / h^2 = 65.5),
refinement with exact solves of that model diverges, while the same with the entries
rounded to FP32 gains about five digits per sweep."""
import numpy as np
import scipy.sparse.linalg as spla

import workloads as W


def _round(a, mantissa_bits):
    """Round FP64 values to nearest-even with the given significand bits (BF16: 8, FP32: 24)."""
    m, e = np.frexp(np.asarray(a, dtype=np.float64))
    scale = 2.0 ** mantissa_bits
    return np.ldexp(np.round(m * scale) / scale, e)


def _refine(S, St, b, sweeps):
    lu = spla.splu(St.tocsc())
    x = np.zeros_like(b)
    res = []
    for _ in range(sweeps):
        r = b - S @ x
        res.append(np.linalg.norm(r) / np.linalg.norm(b))
        x = x + lu.solve(r)
    return res


def test_rounding_helper_matches_float32():
    x = np.random.default_rng(0).standard_normal(1000) * 10.0 ** np.random.default_rng(1).integers(-8, 8, 1000)
    assert np.array_equal(_round(x, 24), x.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(_round(x, 8) - x) <= 2.0 ** -8 * np.abs(x))


def test_bf16_operator_breaks_refinement_at_p4():
    from oracle.solve import LDG
    n, p = 32, 4
    tau = 65.5 / n ** 2
    cV, V0T, side = W.square_mesh(n, jitter=0.2, seed=11)
    bdr = W.boundary_types(side, (2, 4), (1, 3))
    L = LDG(cV, V0T, bdr, p)
    man = W.Manufactured(W.d_config2)
    S = L.operator(L.project(lambda x, y: man.d(0.0, x, y)), tau).tocsr()
    b = S @ L.project(lambda x, y: man.c(tau, x, y)).ravel()
    S16, S32 = S.copy(), S.copy()
    S16.data = _round(S.data, 8)
    S32.data = _round(S.data, 24)
    r32 = _refine(S, S32, b, 3)
    r16 = _refine(S, S16, b, 6)
    assert r32[2] <= 1e-9, r32          # FP32 entries: two sweeps reach the step's tolerance
    assert r16[5] > 1.0, r16            # BF16 entries: the sweeps diverge
