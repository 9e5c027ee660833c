"""The learned warm start: the network kernels (festung_mlp_*) against an FP64 numpy
restatement of the same network, the features against the oracle's residual, and the
guess path of the step (the answer does not depend on the guess)."""
import numpy as np
import pytest

import workloads as W
from helpers import edge_samples, gpu_solver, mesh, samples, smooth_d

pytestmark = pytest.mark.gpu
HID = 64


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _bf16(a):
    """Round FP32 values to BF16 (nearest, ties to even) and back."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _unpack(p, n_in, n_out):
    o = 0
    out = []
    for shape in ((HID, n_in), (HID,), (HID, HID), (HID,), (n_out, HID), (n_out,)):
        size = int(np.prod(shape))
        out.append(p[o:o + size].reshape(shape).astype(np.float64))
        o += size
    W1, b1, W2, b2, W3, b3 = out
    return [_bf16(W1.astype(np.float32)).astype(np.float64), b1, _bf16(W2.astype(np.float32)).astype(np.float64), b2,
            _bf16(W3.astype(np.float32)).astype(np.float64), b3]


def _reference(params, X, T, Wt=None):
    """Loss (1 / 2R) sum (w (y - t))^2 and its gradient in FP64 (BF16-valued weights)."""
    W1, b1, W2, b2, W3, b3 = params
    X = X.astype(np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0)
    Y = h2 @ W3.T + b3
    R = X.shape[0]
    w = np.ones_like(Y) if Wt is None else Wt.astype(np.float64)
    E = w * w * (Y - T) / R
    loss = 0.5 * np.sum((w * (Y - T)) ** 2) / R
    gW3, gb3 = E.T @ h2, E.sum(0)
    d2 = (E @ W3) * (a2 > 0)
    gW2, gb2 = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1, gb1 = d1.T @ X, d1.sum(0)
    grad = np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return Y, loss, grad


def test_mlp_forward_and_gradient_match_fp64_reference():
    import torch
    from paper_1408_3877_gb300 import festung as F
    n_in, n_out, rows = 43, 10, 300
    net = F.MLP(n_in, n_out, seed=3)
    rng = np.random.default_rng(1)
    p0 = rng.normal(0, 0.3, net.n_params).astype(np.float32)   # non-zero biases too
    net.set(p0)
    X = rng.normal(size=(rows, n_in)).astype(np.float32)
    T = rng.normal(size=(rows, n_out)).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    Y = torch.empty(rows, n_out, device="cuda")
    net.forward(Xd, Y)
    loss = net.grad(Xd, Td)
    p, g = net.get()
    assert np.array_equal(p, p0)
    Yr, lr_, gr = _reference(_unpack(p, n_in, n_out), X, T.astype(np.float64))
    assert np.max(np.abs(Y.cpu().numpy() - Yr)) <= 1e-5 * np.max(np.abs(Yr))
    assert abs(loss - lr_) <= 1e-5 * lr_
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr), np.linalg.norm(g - gr) / np.linalg.norm(gr)
    # with per-output weights
    Wt = rng.uniform(0.5, 3.0, size=(rows, n_out)).astype(np.float32)
    loss_w = net.grad(Xd, Td, torch.tensor(Wt, device="cuda"))
    _, gw = net.get()
    _, lw_ref, gw_ref = _reference(_unpack(p, n_in, n_out), X, T.astype(np.float64), Wt)
    assert abs(loss_w - lw_ref) <= 1e-5 * lw_ref
    assert np.linalg.norm(gw - gw_ref) <= 1e-4 * np.linalg.norm(gw_ref)
    net.close()


def test_mlp_adam_step():
    import torch
    from paper_1408_3877_gb300 import festung as F
    net = F.MLP(7, 3, seed=5)
    rng = np.random.default_rng(2)
    X = torch.tensor(rng.normal(size=(64, 7)).astype(np.float32), device="cuda")
    T = torch.tensor(rng.normal(size=(64, 3)).astype(np.float32), device="cuda")
    net.grad(X, T)
    p0, g = net.get()
    lr = 1e-3
    net.adam(lr)
    p1, _ = net.get()
    # first Adam step: m = (1 - b1) g, v = (1 - b2) g^2, bias-corrected update lr g / (|g| + eps)
    want = p0 - lr * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p1 - want)) <= 1e-6
    net.close()


def test_mlp_learns_a_linear_map():
    import torch
    from paper_1408_3877_gb300 import festung as F
    rng = np.random.default_rng(4)
    A = rng.normal(size=(5, 12)) / np.sqrt(12)
    X = rng.normal(size=(4096, 12)).astype(np.float32)
    T = (X @ A.T).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    net = F.MLP(12, 5, seed=1)
    first = net.grad(Xd, Td)
    for _ in range(400):
        net.grad(Xd, Td)
        net.adam(3e-3)
    last = net.grad(Xd, Td)
    assert last < 0.05 * first, (first, last)
    net.close()


def test_features_match_oracle_residual():
    import torch
    from oracle.solve import LDG
    cV, V0T, bdr = mesh(5, "mixed", seed=7)
    p, tau, t = 2, 0.01, 0.01
    man = W.Manufactured(W.d_config2)
    s = gpu_solver(cV, V0T, bdr, p)
    s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
    s.set_coeff(samples(s, smooth_d))
    s.set_source(samples(s, lambda x, y: man.f(t, x, y)))
    s.set_bc(edge_samples(s, lambda x, y: man.c(t, x, y)), edge_samples(s, lambda x, y: man.gN(t, x, y)))
    K, N = s.K, s.N
    X = torch.empty(K, 3 + 4 * N, dtype=torch.float32, device="cuda")
    Wt = torch.empty(K, N, dtype=torch.float32, device="cuda")
    rs = s.warmstart_features(tau, X, Wt)
    X, Wt = X.cpu().numpy(), Wt.cpu().numpy()
    L = LDG(cV, V0T, bdr, p)
    D = L.project(smooth_d)
    C0 = L.project(lambda x, y: man.c(0.0, x, y))
    b = L.rhs(C0, D, L.project(lambda x, y: man.f(t, x, y)), lambda x, y: man.c(t, x, y),
              lambda x, y: man.gN(t, x, y), tau)
    r = (b - L.operator(D, tau) @ C0.ravel()).reshape(K, N)
    q = r / (2 * L.g.areaT)[:, None]    # M^{-1} r, M = 2|T_k| I
    rs_ref = np.sqrt(np.mean(q ** 2))
    assert abs(rs - rs_ref) <= 1e-9 * rs_ref
    order = s.element_order()           # row i of X is the caller's triangle order[i]
    own = X[:, 3:3 + N]
    assert np.max(np.abs(own - (q[order] / rs_ref))) <= 1e-5 * np.max(np.abs(q / rs_ref))
    dmean = np.mean(D[:, 0])
    assert np.max(np.abs(X[:, 0:3] - D[order, 0:3] / dmean)) <= 1e-5
    # loss weights: sqrt of the diagonal of S over 2|T_k| (FP32 blocks)
    dS = L.operator(D, tau).diagonal().reshape(K, N) / (2 * L.g.areaT)[:, None]
    assert np.max(np.abs(Wt - np.sqrt(dS[order])) / np.sqrt(dS[order])) <= 1e-4
    s.close()


def test_exact_guess_needs_no_iterations_and_keeps_the_answer():
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr = mesh(8, "mixed", seed=8)
    man = W.Manufactured(W.d_config2)
    tau, t = 0.005, 0.005
    sols = []
    for guess in (False, True):
        s = gpu_solver(cV, V0T, bdr, 2)
        s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
        C0 = s.get_state()
        s.set_coeff(samples(s, lambda x, y: man.d(t, x, y)))
        s.set_source(samples(s, lambda x, y: man.f(t, x, y)))
        s.set_bc(edge_samples(s, lambda x, y: man.c(t, x, y)), edge_samples(s, lambda x, y: man.gN(t, x, y)))
        if guess:
            s.set_guess(sols[0] - C0)
        info = s.step(tau, tol=1e-11 if guess else 1e-12, prec=F.MIXED)
        sols.append(s.get_state())
        if guess:
            assert info["initial_rel_residual"] <= 1e-10 and info["iterations"] == 0, info
        s.close()
    assert np.linalg.norm(sols[1] - sols[0]) <= 1e-10 * np.linalg.norm(sols[0])
