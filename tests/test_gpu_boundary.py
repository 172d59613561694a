"""The context-level entry points of the C ABI on the GPU:

- lhdm_solve_batched (one persistent launch over uneven instances) against
  lhdm_solve of each instance and the oracle; the second call with the same
  arguments reuses the plan and is replayed from a captured CUDA graph;
- lhdm_backward with an instance index and lhdm_backward_batched against
  the dense closed form (oracle/adjoint.py);
- the NNLS layer (torch.autograd.Function) on a 512 x 1024 instance of the
  layer workload: gradients against the closed form and against central
  differences (h = 1e-6) with the passive set asserted stable;
- failure detection: a grid barrier that can never be released makes every
  bounded wait run out; the solve reports LHDM_ERR_TIMEOUT, the kernel
  returns, and the next solve on the same context matches the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle.adjoint import nnls_adjoint
from paper_2108_05345_gb300 import workloads as WL
from gpu_util import RTOL, assert_parity, dev, solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05345_gb300 import build, lhdm
    build.build()
    return lhdm


def uneven(count=12):
    sizes = WL.batched_sizes()
    idx = list(range(count))
    return [WL.batched_instance(i, min(sizes[i], 200)) for i in idx]


def test_solve_batched_matches_single_and_oracle(L):
    inst = uneven()
    ctx = L.Context(400, 800, max_batch=len(inst))
    dv = [dev(L, A, b) for A, b, _ in inst]
    As, bs = [d[0] for d in dv], [d[1] for d in dv]
    prm = L.default_params(k_max=16)
    xs, ps, infos = ctx.solve_batched(As, bs, prm)
    torch.cuda.synchronize()
    infl = ctx.info_list(infos, len(inst))
    single = L.Context(400, 800)
    for i, (A, b, _) in enumerate(inst):
        x1, p1, _ = single.solve(As[i], bs[i], prm)
        assert torch.equal(p1, ps[i])
        assert float(torch.linalg.norm(x1 - xs[i])) <= RTOL * float(torch.linalg.norm(x1))
        ref = O.nnls(A, b, k_max=16, trace=True)
        p = ps[i].cpu().numpy()
        assert_parity(xs[i].cpu().numpy(), p[p >= 0], infl[i], ref)
    single.close()
    # same arguments: the plan is reused; capture that call and replay it
    first = [x.clone() for x in xs]
    for x in xs:
        x.zero_()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        ctx.solve_batched(As, bs, prm, xs=xs, ps=ps, infos=infos, stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        ctx.solve_batched(As, bs, prm, xs=xs, ps=ps, infos=infos, stream=stream)
    for x in xs:
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, c in zip(first, xs):
        assert torch.equal(a, c)
    # batch beyond max_batch is refused
    with pytest.raises(RuntimeError):
        ctx.solve_batched(As + As[:1], bs + bs[:1], prm)
    ctx.close()


def test_backward_by_index_and_batched(L):
    inst = [WL.layer_batch(count=1, m=120, n=240, s=12, seed0=s)[0] for s in range(5)]
    ctx = L.Context(120, 240, max_batch=len(inst))
    dv = [dev(L, A, b) for A, b, _, _ in inst]
    As, bs = [d[0] for d in dv], [d[1] for d in dv]
    xs, ps, infos = ctx.solve_batched(As, bs, L.default_params(k_max=8))
    torch.cuda.synchronize()
    gs = [2.0 * (x - torch.from_numpy(t).cuda()) for x, (_, _, _, t) in zip(xs, inst)]
    dbs, dAs = ctx.backward_batched(As, gs)
    for i, (A, b, _, xt) in enumerate(inst):
        x = xs[i].cpu().numpy()
        p = ps[i].cpu().numpy()
        ref_db, ref_dA = nnls_adjoint(A, b, x, p[p >= 0], gs[i].cpu().numpy())
        db1, dA1 = ctx.backward(As[i], gs[i], idx=i)
        torch.cuda.synchronize()
        for db, dA in ((dbs[i], dAs[i]), (db1, dA1)):
            assert np.linalg.norm(db.cpu().numpy() - ref_db) <= 1e-9 * np.linalg.norm(ref_db)
            assert np.linalg.norm(dA.cpu().numpy() - ref_dA) <= 1e-9 * np.linalg.norm(ref_dA)
    with pytest.raises(RuntimeError):
        ctx.backward(As[0], gs[0], idx=len(inst))
    ctx.close()


def test_layer_gradients_layer_size(L):
    from paper_2108_05345_gb300.layer import NNLSLayer
    A, b, _, xt = WL.layer_batch(count=1, seed0=5)[0]
    m, n = A.shape
    layer = NNLSLayer(m, n, k_max=32)
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    xtt = torch.from_numpy(xt).cuda()
    x = layer(At, bt)
    loss = ((x - xtt) ** 2).sum()
    loss.backward()
    xs = x.detach().cpu().numpy()
    ref = O.nnls(A, b, k_max=32)
    assert np.linalg.norm(xs - ref["x"]) <= RTOL * np.linalg.norm(ref["x"])
    P = np.flatnonzero(xs > 0)
    ref_db, ref_dA = nnls_adjoint(A, b, xs, P, 2.0 * (xs - xt))
    gb, gA = bt.grad.cpu().numpy(), At.grad.cpu().numpy()
    assert np.linalg.norm(gb - ref_db) <= 1e-9 * np.linalg.norm(ref_db)
    assert np.linalg.norm(gA - ref_dA) <= 1e-9 * np.linalg.norm(ref_dA)
    # central differences through the layer (h = 1e-6), passive set stable
    h = 1e-6

    def f(Ah, bh):
        with torch.no_grad():
            xx = layer(torch.from_numpy(np.ascontiguousarray(Ah)).cuda(), torch.from_numpy(bh).cuda())
        xx = xx.cpu().numpy()
        assert np.flatnonzero(xx > 0).tolist() == P.tolist()
        return float(np.sum((xx - xt) ** 2))

    for i in (0, 100, 511):
        e = np.zeros(m)
        e[i] = h
        fd = (f(A, b + e) - f(A, b - e)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gb[i])
    for (i, j) in [(3, P[0]), (200, P[len(P) // 2]), (510, P[-1])]:
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (f(A + E, b) - f(A - E, b)) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-6 * max(1.0, abs(fd)), (i, j, fd, gA[i, j])


def test_layer_batched(L):
    from paper_2108_05345_gb300.layer import NNLSLayer
    inst = WL.layer_batch(count=4, seed0=20)
    m, n = inst[0][0].shape
    layer = NNLSLayer(m, n, max_batch=4, k_max=32)
    A = torch.from_numpy(np.stack([a for a, _, _, _ in inst])).cuda().requires_grad_(True)
    b = torch.from_numpy(np.stack([v for _, v, _, _ in inst])).cuda().requires_grad_(True)
    xt = torch.from_numpy(np.stack([t for _, _, _, t in inst])).cuda()
    x = layer(A, b)
    ((x - xt) ** 2).sum().backward()
    for i, (Ai, bi, _, ti) in enumerate(inst):
        xs = x[i].detach().cpu().numpy()
        P = np.flatnonzero(xs > 0)
        ref_db, ref_dA = nnls_adjoint(Ai, bi, xs, P, 2.0 * (xs - ti))
        assert np.linalg.norm(b.grad[i].cpu().numpy() - ref_db) <= 1e-9 * np.linalg.norm(ref_db)
        assert np.linalg.norm(A.grad[i].cpu().numpy() - ref_dA) <= 1e-9 * np.linalg.norm(ref_dA)


def test_bounded_wait_runs_out_and_context_recovers(L):
    A, b, _ = WL.overdetermined_uniform(3, m=600, n=300)
    ctx = L.Context(600, 300)
    At, bt = dev(L, A, b)
    ctx.set_wait_limit(20_000_000)  # 20 ms
    ctx.stall_next_solve()
    x, p, info = ctx.solve(At, bt, L.default_params(k_max=16))
    assert info["status"] == L.LHDM_ERR_TIMEOUT
    ctx.set_wait_limit(0)  # back to the default bound
    x, P, _, info = solve(L, ctx, A, b, k_max=16)
    ref = O.nnls(A, b, k_max=16, trace=True)
    assert_parity(x, P, info, ref, trace=ctx.trace())
    ctx.close()
