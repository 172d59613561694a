"""CUDA path vs the CPU oracle at the benchmarked sizes, in the launch
configurations bench.py times, and the rank-guard cases.

- 4096 x 2048 overdetermined problem at k_max 16 and 64 (k_max 1 and 32 are
  in test_gpu_parity.py);
- the 2048 x 8192 sparse-recovery sweep at s = 64, 512 (against x0 and the
  oracle) and s = 1024 (beyond the recovery threshold: zero residual with a
  non-unique minimiser, so checked by the optimality conditions, which hold
  at any size);
- the batched uneven workload up to m = 512: at least eight instances of
  every size bucket, the largest included, in one persistent launch with
  k_max per bucket, each against the oracle at the same k_max;
- the adjoint on instances of the layer workload (512 x 1024) against the
  dense closed form on the final passive set, and central differences
  (h = 1e-6) through the solve on one of them;
- the rank guard: a DM block with a dependent column, and exact duplicates.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle.adjoint import nnls_adjoint
from paper_2108_05345_gb300 import workloads as WL
from gpu_util import RTOL, TIE, assert_parity, dev, kkt, significant, solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05345_gb300 import build, lhdm
    build.build()
    return lhdm


@pytest.fixture(scope="module")
def ctx(L):
    c = L.Context(4096, 8192)
    yield c
    c.close()


@pytest.mark.parametrize("k_max", [16, 64])
def test_overdetermined_full_size(L, ctx, k_max):
    A, b, _ = WL.overdetermined_uniform(0)
    x, P, _, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max)
    assert_parity(x, P, info, ref, counters=False)


@pytest.mark.parametrize("s", [64, 512])
def test_sparse_sweep_against_oracle(L, ctx, s):
    A, b, x0 = WL.sparse_recovery_sweep(0, s)
    x, P, _, info = solve(L, ctx, A, b, k_max=64)
    ref = O.nnls(A, b, k_max=64, trace=True)
    assert info["status"] == 0
    # recovery of x0 (noiseless, below the recovery threshold)
    assert np.linalg.norm(x - x0) <= RTOL * np.linalg.norm(x0)
    assert significant(x) == np.flatnonzero(x0).tolist()
    assert np.linalg.norm(x - ref["x"]) <= RTOL * np.linalg.norm(ref["x"])
    if not (ref["trace_margin"] < TIE).any():
        assert P.tolist() == ref["passive"].tolist()


def test_sparse_sweep_beyond_threshold(L, ctx):
    """s = 1024 of m = 2048: b = A x0 has many nonnegative representations;
    the solve must end at an optimal point: x >= 0, residual ~ 0, and the
    dual w = A^T r below tol_w on the zero set (KKT)."""
    A, b, x0 = WL.sparse_recovery_sweep(0, 1024)
    x, P, _, info = solve(L, ctx, A, b, k_max=64)
    assert info["status"] == 0
    xmin, wz, wp = kkt(A, b, x, info["tol_w"])
    assert xmin >= 0.0
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    assert wz <= 10 * info["tol_w"] and wp <= 10 * info["tol_w"]
    assert set(np.flatnonzero(x).tolist()) <= set(P.tolist())


def batch_sample(per_bucket=8):
    """Indices of the 1024-instance batched workload: per_bucket instances of
    every size bucket of n (n <= 128, <= 256, <= 512, <= 1024), the largest
    instance of each bucket first."""
    sizes = np.array(WL.batched_sizes())
    n = 2 * sizes
    edges = [0, 128, 256, 512, 1024]
    picks = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        idx = np.flatnonzero((n > lo) & (n <= hi))
        order = idx[np.argsort(-sizes[idx], kind="stable")]
        picks += [int(order[0])] + [int(i) for i in order[1:][:: max(1, len(order) // per_bucket)][: per_bucket - 1]]
    return picks


def test_batched_up_to_m512(L):
    picks = batch_sample()
    sizes = WL.batched_sizes()
    assert max(sizes[i] for i in picks) == 512
    inst = [WL.batched_instance(i, sizes[i]) for i in picks]
    dv = [dev(L, A, b) for A, b, _ in inst]
    batch = L.Batch([d[0] for d in dv], [d[1] for d in dv], L.default_params(k_max=0))
    batch.run()
    torch.cuda.synchronize()
    infos = batch.info()
    for i, (A, b, _) in enumerate(inst):
        k = batch.kmax(i)
        ref = O.nnls(A, b, k_max=k, trace=True)
        p = batch.ps[i].cpu().numpy()
        assert_parity(batch.xs[i].cpu().numpy(), p[p >= 0], infos[i], ref)
    batch.close()


def test_adjoint_layer_size(L):
    inst = WL.layer_batch(count=4)
    m, n = inst[0][0].shape
    ctx = L.Context(m, n)
    prm = L.default_params(k_max=32)
    for A, b, _, xt in inst:
        At, bt = dev(L, A, b)
        x, p, info = ctx.solve(At, bt, prm)
        assert info["status"] == 0
        xs = x.cpu().numpy()
        P = p.cpu().numpy()
        P = P[P >= 0]
        g = 2.0 * (xs - xt)
        db, dA = ctx.backward(At, torch.from_numpy(g).cuda())
        ref_db, ref_dA = nnls_adjoint(A, b, xs, P, g)
        assert np.linalg.norm(db.cpu().numpy() - ref_db) <= 1e-9 * np.linalg.norm(ref_db)
        assert np.linalg.norm(dA.cpu().numpy() - ref_dA) <= 1e-9 * np.linalg.norm(ref_dA)
        ref = O.nnls(A, b, k_max=32)
        assert np.linalg.norm(xs - ref["x"]) <= RTOL * np.linalg.norm(ref["x"])
    ctx.close()


@pytest.mark.parametrize("seed", range(4))
def test_rank_guard_dependent_block(L, ctx, seed):
    """The oracle's hand-derived case (tests/test_oracle.py): J = {a6, a1, a4}
    with a6 = a1 + a4 is cut to two columns by the rank guard."""
    A, b, (i1, i2, i3) = WL.dependent_triple(seed=seed)
    x, P, _, info = solve(L, ctx, A, b, k_max=8, tau1=0.4)
    ref = O.nnls(A, b, k_max=8, tau1=0.4, trace=True)
    assert ctx.trace()[0].tolist() == [3, 2, 0, 2, 0, i3]
    assert P.tolist() == sorted([i1, i3]) and info["n_drop"] == 0 and info["n_outer"] == 1
    assert_parity(x, P, info, ref, trace=ctx.trace())


@pytest.mark.parametrize("k_max", [1, 4])
@pytest.mark.parametrize("where", ["after", "before"])
def test_duplicate_column(L, ctx, k_max, where):
    for seed in range(6):
        A, b = WL.tiny(seed, 12, 8)
        base = O.nnls(A, b, k_max=k_max)
        c = base["passive"].tolist()[0]
        at = A.shape[1] if where == "after" else c
        A2 = WL.with_duplicate(A, c, at)
        x, P, _, info = solve(L, ctx, A2, b, k_max=k_max)
        ref = O.nnls(A2, b, k_max=k_max, trace=True)
        assert_parity(x, P, info, ref, trace=ctx.trace())
