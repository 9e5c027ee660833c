"""Batches of independent problems (festung_batch_*): every problem of a batch step must
match the same problem stepped alone (FP64 path, itself pinned to the oracle's solve of
eq. fullSystem) and meet the tolerance on its own residual, with the problems joined
into one mesh per group (FESTUNG_BATCH_UNION) or stepped one each by several workers
(FESTUNG_BATCH_CONCURRENT)."""
import numpy as np
import pytest

import workloads as W
from helpers import edge_samples, gpu_solver, samples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _dfun(a, b):
    def d(t, x, y):
        s, c = np.sin(a * x), np.cos(b * y)
        return 1.0 + 0.4 * s * c, 0.4 * a * np.cos(a * x) * c, -0.4 * b * s * np.sin(b * y)
    return d


PROBLEMS = [(6, 1, 1.0, 2.0), (9, 2, 3.0, 1.0), (7, 3, 2.0, 2.0), (12, 1, 4.0, 3.0), (8, 2, 1.5, 2.5),
            (5, 3, 2.5, 1.0)]


def _make(n, p, a, b, seed):
    cV, V0T, side = W.square_mesh(n, jitter=0.2, seed=seed)
    bdr = W.boundary_types(side, (1, 2, 3, 4), ())
    return cV, V0T, bdr, W.Manufactured(_dfun(a, b))


def _load(s, man, t):
    s.set_coeff(samples(s, lambda x, y: man.d(t, x, y)))
    s.set_source(samples(s, lambda x, y: man.f(t, x, y)))
    s.set_bc(edge_samples(s, lambda x, y: man.c(t, x, y)), None)


@pytest.mark.parametrize("mode,workers,user_stream", [("BATCH_UNION", 0, False), ("BATCH_CONCURRENT", 3, False),
                                                     ("BATCH_CONCURRENT", 0, True)])
def test_batch_matches_single_problem_steps(mode, workers, user_stream):
    import torch
    from paper_1408_3877_gb300 import festung as F
    tau, steps = 0.005, 3
    probs = [_make(n, p, a, b, seed=10 + q) for q, (n, p, a, b) in enumerate(PROBLEMS)]
    bs, ss = [], []
    for (cV, V0T, bdr, man), (n, p, a, b) in zip(probs, PROBLEMS):
        for lst in (bs, ss):
            s = gpu_solver(cV, V0T, bdr, p)
            s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
            lst.append(s)
    batch = F.Batch(bs)
    batch.set_mode(getattr(F, mode), workers)
    stream = torch.cuda.Stream() if user_stream else None
    if stream is not None:
        batch.set_stream(stream)
    for k in range(1, steps + 1):
        t = k * tau
        for s, (_, _, _, man) in zip(bs, probs):
            _load(s, man, t)
        l0 = batch.launch_count()
        infos = batch.step(tau, tol=1e-12, inner_tol=1e-2)
        if stream is not None:
            stream.synchronize()
        assert batch.launch_count() > l0
        for q, (s, (_, _, _, man)) in enumerate(zip(ss, probs)):
            _load(s, man, t)
            s.step(tau, tol=1e-13, prec=F.FP64)
            Cs, Cb = s.get_state(), bs[q].get_state()
            err = np.linalg.norm(Cb - Cs) / np.linalg.norm(Cs)
            assert err <= 1e-9, (k, q, err, infos[q])
            assert infos[q]["rel_residual"] <= 1e-12, infos[q]
    assert batch.launch_count() > 0
    batch.close()
    for s in bs + ss:
        s.close()


@pytest.mark.parametrize("mode", ["BATCH_UNION", "BATCH_CONCURRENT"])
def test_batch_restarts_history_after_outside_state_change(mode):
    from paper_1408_3877_gb300 import festung as F
    tau = 0.005
    (n, p, a, b) = PROBLEMS[1]
    cV, V0T, bdr, man = _make(n, p, a, b, seed=3)
    (n2, p2, a2, b2) = PROBLEMS[4]
    cV2, V0T2, bdr2, man2 = _make(n2, p2, a2, b2, seed=4)
    s1, s2 = gpu_solver(cV, V0T, bdr, p), gpu_solver(cV2, V0T2, bdr2, p2)
    ref = gpu_solver(cV, V0T, bdr, p)
    for s, m in ((s1, man), (s2, man2), (ref, man)):
        s.set_state(samples(s, lambda x, y: m.c(0.0, x, y)), is_samples=True)
    batch = F.Batch([s1, s2])
    batch.set_mode(getattr(F, mode))
    for k in (1, 2):
        _load(s1, man, k * tau), _load(s2, man2, k * tau)
        batch.step(tau, tol=1e-12)
    # the caller resets problem 1: the batch must not extrapolate from its old states
    C0 = samples(s1, lambda x, y: man.c(0.0, x, y))
    s1.set_state(C0, is_samples=True)
    ref.set_state(C0, is_samples=True)
    _load(s1, man, 3 * tau), _load(s2, man2, 3 * tau), _load(ref, man, 3 * tau)
    info = batch.step(tau, tol=1e-12)
    ref.step(tau, tol=1e-13, prec=F.FP64)
    err = np.linalg.norm(s1.get_state() - ref.get_state()) / np.linalg.norm(ref.get_state())
    assert err <= 1e-9, (err, info)
    batch.close()
    for s in (s1, s2, ref):
        s.close()


def test_batch_rejects_bad_members():
    from paper_1408_3877_gb300 import festung as F
    cV, V0T, bdr, _ = _make(4, 1, 1.0, 1.0, seed=1)
    s = gpu_solver(cV, V0T, bdr, 1)
    raw = F.Solver(cV, V0T, bdr)  # not set up
    with pytest.raises(F.FestungError) as e:
        F.Batch([s, raw])
    assert e.value.code == F.ESTATE
    with pytest.raises(F.FestungError) as e:
        F.Batch([s, s])
    assert e.value.code == F.EINVAL
    b = F.Batch([s])
    for mode, workers in ((2, 0), (F.BATCH_CONCURRENT, -1), (F.BATCH_CONCURRENT, 65)):
        with pytest.raises(F.FestungError) as e:
            b.set_mode(mode, workers)
        assert e.value.code == F.EINVAL
    b.close()
    s.close()
    raw.close()


@pytest.mark.parametrize("mode", ["BATCH_UNION", "BATCH_CONCURRENT"])
def test_batch_members_match_oracle(mode):
    """Every member of a batch step against the oracle's sparse direct solve of its own
    eliminated system (Sec. 2.5) from the same state: within 1e-9 relative L2 at tolerance
    1e-12.  One member (24 x 24, 1,152 triangles) spans several tiles of its own."""
    from oracle.solve import LDG
    from paper_1408_3877_gb300 import festung as F
    tau, t = 0.005, 0.005
    specs = PROBLEMS[:4] + [(24, 2, 2.0, 3.0)]
    probs = [_make(n, p, a, b, seed=30 + q) for q, (n, p, a, b) in enumerate(specs)]
    bs = []
    for (cV, V0T, bdr, man), (n, p, a, b) in zip(probs, specs):
        s = gpu_solver(cV, V0T, bdr, p)
        s.set_state(samples(s, lambda x, y: man.c(0.0, x, y)), is_samples=True)
        _load(s, man, t)
        bs.append(s)
    batch = F.Batch(bs)
    batch.set_mode(getattr(F, mode), 0)
    infos = batch.step(tau, tol=1e-12, inner_tol=1e-2)
    for q, ((cV, V0T, bdr, man), (n, p, a, b)) in enumerate(zip(probs, specs)):
        L = LDG(cV, V0T, bdr, p)
        Co = L.step(L.project(lambda x, y: man.c(0.0, x, y)), L.project(lambda x, y: man.d(t, x, y)),
                    L.project(lambda x, y: man.f(t, x, y)), lambda x, y: man.c(t, x, y), None, tau)
        Cb = bs[q].get_state()
        err = np.linalg.norm(Cb - Co) / np.linalg.norm(Co)
        assert err <= 1e-9, (q, err, infos[q])
        assert infos[q]["rel_residual"] <= 1e-12, infos[q]
    batch.close()
    for s in bs:
        s.close()
