"""Batched persistent solves and the adjoint, CUDA path vs the CPU oracle.

Batched: every instance of one launch against an oracle solve of the same
instance with the same k_max (identical sorted passive set, rel err
<= 1e-10); a rounding tie in the oracle's path (decision margin < 1e-9)
relaxes the passive-set check to the significant support.  The launch is
also replayed from a captured CUDA graph.

Adjoint: dL/db and dL/dA against the dense closed form on the final passive
set (oracle/adjoint.py) and against central differences of the GPU solve.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle.adjoint import nnls_adjoint
from paper_2108_05345_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
RTOL = 1e-10
TIE = 1e-9


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05345_gb300 import build, lhdm
    build.build()
    return lhdm


def to_dev(L, A, b):
    At = L.colmajor(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    return At, torch.from_numpy(np.ascontiguousarray(b)).cuda()


def check_instance(x, P, info, ref):
    assert info["status"] == ref["status"] == 0
    tied = (ref["trace_margin"] < TIE).any() if len(ref["trace_margin"]) else False
    if tied:
        sig = lambda v: np.flatnonzero(v > 1e-9 * max(np.abs(v).max(), 1e-300)).tolist()
        assert sig(x) == sig(ref["x"])
    else:
        assert P.tolist() == ref["passive"].tolist()
        assert (info["n_outer"], info["n_inner"], info["n_drop"]) == (ref["n_outer"], ref["n_inner"], ref["n_drop"])
    nx = np.linalg.norm(ref["x"])
    assert np.linalg.norm(x - ref["x"]) <= RTOL * max(nx, 1e-300)


def make_batch(count, m_hi, seed=0):
    inst = WL.batched_uneven(batch_seed=seed, count=count, m_lo=64, m_hi=m_hi)
    return [(A, b) for A, b, _ in inst]


@pytest.mark.parametrize("k_max", [1, 16, 0])
def test_batched_matches_oracle(L, k_max):
    inst = make_batch(24, 200)
    dev = [to_dev(L, A, b) for A, b in inst]
    batch = L.Batch([d[0] for d in dev], [d[1] for d in dev], L.default_params(k_max=k_max))
    batch.run()
    torch.cuda.synchronize()
    infos = batch.info()
    for i, (A, b) in enumerate(inst):
        k = batch.kmax(i)
        assert k == (k_max if k_max > 0 else k)
        ref = O.nnls(A, b, k_max=k, trace=True)
        x = batch.xs[i].cpu().numpy()
        p = batch.ps[i].cpu().numpy()
        check_instance(x, p[p >= 0], infos[i], ref)
        assert (p[len(p[p >= 0]):] == -1).all()
    batch.close()


def test_batched_repeat_and_graph_replay(L):
    inst = make_batch(16, 160, seed=3)
    dev = [to_dev(L, A, b) for A, b in inst]
    batch = L.Batch([d[0] for d in dev], [d[1] for d in dev], L.default_params(k_max=8))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(stream)
    torch.cuda.synchronize()
    first = [x.cpu().numpy().copy() for x in batch.xs]
    for x in batch.xs:
        x.zero_()
    # capture the single persistent launch and replay it
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.run(stream)
    g.replay()
    torch.cuda.synchronize()
    for x0, x in zip(first, batch.xs):
        assert np.array_equal(x0, x.cpu().numpy())
    batch.close()


def test_batched_edge_sizes(L):
    shapes = [(1, 1), (1, 5), (5, 1), (3, 7), (64, 128), (130, 65)]
    inst = [WL.tiny(100 + i, m, n) for i, (m, n) in enumerate(shapes)]
    dev = [to_dev(L, A, b) for A, b in inst]
    batch = L.Batch([d[0] for d in dev], [d[1] for d in dev], L.default_params(k_max=4))
    batch.run()
    torch.cuda.synchronize()
    infos = batch.info()
    for i, (A, b) in enumerate(inst):
        ref = O.nnls(A, b, k_max=4, trace=True)
        p = batch.ps[i].cpu().numpy()
        check_instance(batch.xs[i].cpu().numpy(), p[p >= 0], infos[i], ref)
    batch.close()


def layer_instance(seed, m=60, n=100, s=6):
    rng = np.random.default_rng(seed)
    A = rng.normal(0, 1 / np.sqrt(m), size=(m, n))
    x0 = np.zeros(n)
    x0[rng.choice(n, s, replace=False)] = rng.uniform(0.5, 1.0, s)
    b = A @ x0 + 1e-3 * rng.normal(size=m)
    xt = x0 + 1e-2 * rng.normal(size=n)
    return np.asfortranarray(A), b, xt


def test_adjoint_closed_form_and_fd(L):
    A, b, xt = layer_instance(1)
    m, n = A.shape
    ctx = L.Context(m, n)
    At, bt = to_dev(L, A, b)
    prm = L.default_params(k_max=8)
    x, p, info = ctx.solve(At, bt, prm)
    xs = x.cpu().numpy()
    P = p.cpu().numpy()
    P = P[P >= 0]
    g = 2.0 * (xs - xt)
    db, dA = ctx.backward(At, torch.from_numpy(g).cuda())
    db = db.cpu().numpy()
    dA = dA.cpu().numpy()
    ref_db, ref_dA = nnls_adjoint(A, b, xs, P, g)
    assert np.linalg.norm(db - ref_db) <= 1e-9 * np.linalg.norm(ref_db)
    assert np.linalg.norm(dA - ref_dA) <= 1e-9 * np.linalg.norm(ref_dA)
    Z = np.setdiff1d(np.arange(n), P)
    assert not dA[:, Z].any()
    # central differences of the GPU solve (h = 1e-6) on a stable passive set
    h = 1e-6

    def loss(Ah, bh):
        Ad, bd = to_dev(L, Ah, bh)
        xx, pp, _ = ctx.solve(Ad, bd, prm)
        pp = pp.cpu().numpy()
        assert pp[pp >= 0].tolist() == P.tolist()
        return float(np.sum((xx.cpu().numpy() - xt) ** 2))

    for i in (0, 7, 31):
        e = np.zeros(m)
        e[i] = h
        fd = (loss(A, b + e) - loss(A, b - e)) / (2 * h)
        assert abs(fd - db[i]) <= 1e-6 * max(1.0, abs(fd))
    for (i, j) in [(3, P[0]), (11, P[-1])]:
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (loss(A + E, b) - loss(A - E, b)) / (2 * h)
        assert abs(fd - dA[i, j]) <= 1e-6 * max(1.0, abs(fd))
    ctx.close()


def test_batched_adjoint(L):
    items = [layer_instance(10 + i, m=50 + 7 * i, n=90 + 5 * i) for i in range(6)]
    dev = [to_dev(L, A, b) for A, b, _ in items]
    batch = L.Batch([d[0] for d in dev], [d[1] for d in dev], L.default_params(k_max=8))
    batch.run()
    torch.cuda.synchronize()
    gs = []
    for i, (A, b, xt) in enumerate(items):
        gs.append(torch.from_numpy(2.0 * (batch.xs[i].cpu().numpy() - xt)).cuda())
    dbs, dAs = batch.backward(gs)
    torch.cuda.synchronize()
    for i, (A, b, xt) in enumerate(items):
        xs = batch.xs[i].cpu().numpy()
        p = batch.ps[i].cpu().numpy()
        ref_db, ref_dA = nnls_adjoint(A, b, xs, p[p >= 0], gs[i].cpu().numpy())
        assert np.linalg.norm(dbs[i].cpu().numpy() - ref_db) <= 1e-9 * np.linalg.norm(ref_db)
        assert np.linalg.norm(dAs[i].cpu().numpy() - ref_dA) <= 1e-9 * np.linalg.norm(ref_dA)
    batch.close()
