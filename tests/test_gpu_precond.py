"""The block-Jacobi preconditioner against the oracle.  The build (k_blockdiag) computes
the N x N diagonal blocks S_kk of the step operator of (E1), S = M + tau (eta (S + S_D)
- sum_m A_m M^{-1} B_m), in FP32; the oracle's blocks are those of its assembled FP64
operator (Sec. 2.5 with z eliminated).  Each GPU block must match to 1e-4 relative
(Frobenius), far below the O(1) change a dropped or mis-signed term makes at tau = 0.01
on this mesh.  The inverses (k_blockinv, FP32 Gauss-Jordan stored in BF16) must give
|P_k S_kk - I| <= (3 * 2^-9 + 1e-4) |P_k| |S_kk| elementwise: BF16 rounding of each
entry (at most 2^-9 relative) and the FP32 build's error, nothing more."""
import numpy as np
import pytest

from helpers import gpu_solver, mesh, samples, smooth_d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mix", ["dirichlet", "neumann", "mixed"])
def test_precond_blocks_match_oracle(p, mix):
    from oracle.solve import LDG
    cV, V0T, bdr = mesh(5, mix, seed=3)
    tau = 0.01
    L = LDG(cV, V0T, bdr, p)
    S = L.operator(L.project(smooth_d), tau).toarray()
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_coeff(samples(s, smooth_d))
    blocks, inv = s.precond_blocks(tau)
    K, N = s.K, s.N
    worst = 0.0
    for k in range(K):
        Skk = S[k * N:(k + 1) * N, k * N:(k + 1) * N]
        err = np.linalg.norm(blocks[k] - Skk) / np.linalg.norm(Skk)
        worst = max(worst, err)
        E = np.abs(inv[k] @ Skk - np.eye(N))
        bound = (3 * 2.0 ** -9 + 1e-4) * (np.abs(inv[k]) @ np.abs(Skk)) + 1e-12
        assert np.all(E <= bound), (k, float(np.max(E / bound)))
    assert worst <= 1e-4, worst
    s.close()
