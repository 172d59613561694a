"""CUDA path vs the CPU oracle, element by element, on seeded inputs.

Bar: identical sorted passive set (index work, bit-exact) and
||x - x_oracle|| / ||x_oracle|| <= 1e-10 (FP64 throughout); the iteration
counters are compared too, since both sides take the same decisions.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2108_05345_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
RTOL = 1e-10


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


def dev(A, b):
    At = torch.from_numpy(np.asfortranarray(A)).cuda()
    At = At.t().contiguous().t() if At.stride(0) != 1 else At
    return At, torch.from_numpy(np.ascontiguousarray(b)).cuda()


def solve(L, ctx, A, b, **kw):
    At, bt = dev(A, b)
    x, p, info = ctx.solve(At, bt, L.default_params(**kw))
    torch.cuda.synchronize()
    ps = p.cpu().numpy()
    return x.cpu().numpy(), ps[ps >= 0], ps, info


# A decision whose comparison is this close to flipping (relative) is taken
# by rounding; from that step on only the (unique) final result is compared.
TIE = 1e-9


def first_divergence(tr_gpu, tr_ref, margin):
    for s in range(min(len(tr_gpu), len(tr_ref))):
        if margin[s] < TIE:
            return None  # step s took a decision by rounding: paths may part here
        if not np.array_equal(tr_gpu[s], tr_ref[s]):
            return s, tr_gpu[s].tolist(), tr_ref[s].tolist()
    if len(tr_gpu) != len(tr_ref):
        return len(tr_ref), None, None
    return None


def assert_parity(x, P, info, ref, counters=True, ctx=None):
    assert info["status"] == ref["status"], (info, ref["status"])
    tied = "trace_margin" in ref and (ref["trace_margin"] < TIE).any()
    if counters and ctx is not None and "trace" in ref:
        d = first_divergence(ctx.trace(), ref["trace"], ref["trace_margin"])
        assert d is None, "decision trace diverges at outer step %s: gpu %s oracle %s" % d
    counters = counters and not tied
    if tied:
        # a rounding tie may leave columns whose coefficient is at the
        # rounding level on one side only: compare the significant support
        sig = lambda v: np.flatnonzero(v > 1e-9 * max(np.abs(v).max(), 1e-300)).tolist()
        assert sig(x) == sig(ref["x"])
    else:
        assert P.tolist() == ref["passive"].tolist()
    nx = max(np.linalg.norm(ref["x"]), 1e-300)
    assert np.linalg.norm(x - ref["x"]) <= RTOL * nx or np.linalg.norm(ref["x"]) == 0 and not x.any()
    if not tied:
        assert info["n_passive"] == ref["n_passive"]
    if counters:
        assert (info["n_outer"], info["n_inner"], info["n_drop"]) == (ref["n_outer"], ref["n_inner"], ref["n_drop"])
    assert abs(info["resid_norm"] - ref["resid_norm"]) <= 1e-9 * max(1.0, ref["resid_norm"])


@pytest.mark.parametrize("k_max", [1, 8, 32])
@pytest.mark.parametrize("seed", range(4))
def test_small_recovery(L, ctx, seed, k_max):
    A, b, x0 = WL.small_recovery(seed)
    x, P, ps, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max, trace=True)
    assert_parity(x, P, info, ref, ctx=ctx)
    sig = np.flatnonzero(x > 1e-9 * np.abs(x).max()).tolist()
    assert sig == np.flatnonzero(x0).tolist()
    assert (ps[len(P):] == -1).all()


@pytest.mark.parametrize("k_max", [1, 16, 64])
def test_overdetermined_with_removals(L, ctx, k_max):
    A, b, _ = WL.overdetermined_uniform(3, m=700, n=350)
    x, P, _, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max, trace=True)
    assert ref["n_inner"] > 0  # the Givens downdate is exercised
    assert_parity(x, P, info, ref, ctx=ctx)


@pytest.mark.parametrize("shape", [(257, 131), (131, 257), (100, 333), (33, 1), (1, 7), (2, 2), (65, 64), (64, 65)])
@pytest.mark.parametrize("k_max", [1, 4, 64])
def test_ragged_shapes(L, ctx, shape, k_max):
    m, n = shape
    A, b = WL.tiny(m * 1000 + n, m, n)
    x, P, _, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max, trace=True)
    assert_parity(x, P, info, ref, ctx=ctx)


@pytest.mark.parametrize("rr,cc,k_max", [(6, 0, 12), (6, 0, 32), (4, 4, 32)])
def test_badly_scaled_rows_and_columns(L, ctx, rr, cc, k_max):
    """Rows scaled by 2^-rr .. 2^rr and columns by 2^-cc .. 2^cc: the blocked
    commit cuts its operands into digits under row and column scales, so
    magnitudes that differ by thousands within one product are its hardest
    case (the scaling itself is exact)."""
    A, b, _ = WL.overdetermined_uniform(5, m=700, n=350)
    rng = np.random.default_rng(11)
    rs = 2.0 ** rng.integers(-rr, rr + 1, size=A.shape[0])
    cs = 2.0 ** rng.integers(-cc, cc + 1, size=A.shape[1])
    A = A * rs[:, None] * cs[None, :]
    b = b * rs
    x, P, _, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max, trace=True)
    assert ref["status"] == 0
    assert_parity(x, P, info, ref, ctx=ctx)


def test_empty_problems(L, ctx):
    for (m, n) in [(0, 5), (5, 0), (0, 0)]:
        A = np.zeros((m, n))
        b = np.ones(m)
        At = torch.zeros((max(m, 1), max(n, 1)), dtype=torch.float64, device="cuda")
        At = L.colmajor(At)[:m, :n]
        bt = torch.ones(max(m, 1), dtype=torch.float64, device="cuda")[:m]
        x, p, info = ctx.solve(At, bt, L.default_params(k_max=4))
        assert info["status"] == 0 and info["n_passive"] == 0
        assert not x.cpu().numpy().any()


@pytest.mark.parametrize("shape", [(8, 12), (12, 8)])
def test_brute_force_sizes(L, ctx, shape):
    m, n = shape
    for seed in range(30):
        A, b = WL.tiny(seed, m, n)
        for k in (1, 4):
            x, P, _, info = solve(L, ctx, A, b, k_max=k)
            ref = O.nnls(A, b, k_max=k, trace=True)
            assert_parity(x, P, info, ref, ctx=ctx)


def test_status_paths(L, ctx):
    A, b, _ = WL.small_recovery(1)
    A2 = A.copy()
    A2[5, 9] = np.nan
    x, P, _, info = solve(L, ctx, A2, b, k_max=8)
    assert info["status"] == L.LHDM_ERR_NONFINITE and len(P) == 0 and not x.any()
    x, P, _, info = solve(L, ctx, A, b, k_max=1, max_outer=3)
    ref = O.nnls(A, b, k_max=1, max_outer=3)
    assert info["status"] == L.LHDM_ERR_MAX_ITER == ref["status"]
    assert info["n_outer"] == 3


def test_tau1_one_no_drops(L, ctx):
    A, b, _ = WL.overdetermined_uniform(5, m=500, n=250)
    x, P, _, info = solve(L, ctx, A, b, k_max=16, tau1=1.0, tau2=0.5)
    ref = O.nnls(A, b, k_max=16, tau1=1.0, tau2=0.5, trace=True)
    assert info["n_drop"] == 0
    assert_parity(x, P, info, ref, ctx=ctx)


def test_feasibility_drops_path(L, ctx):
    # aggressive thresholds make the DM block large enough for drops
    found = False
    for seed in range(6):
        A, b, _ = WL.overdetermined_uniform(seed, m=300, n=200)
        ref = O.nnls(A, b, k_max=64, tau1=0.05, tau2=0.05, delta=0.99, trace=True)
        x, P, _, info = solve(L, ctx, A, b, k_max=64, tau1=0.05, tau2=0.05, delta=0.99)
        assert_parity(x, P, info, ref, ctx=ctx)
        found |= ref["n_drop"] > 0
    assert found


def test_host_buffer_path(L, ctx):
    A, b, _ = WL.overdetermined_uniform(7, m=400, n=300)
    x, p, info = ctx.solve_host(A, b, L.default_params(k_max=16))
    ref = O.nnls(A, b, k_max=16)
    assert_parity(x, p[p >= 0], info, ref)


def test_repeated_solves_are_deterministic(L, ctx):
    A, b, _ = WL.overdetermined_uniform(8, m=600, n=400)
    outs = [solve(L, ctx, A, b, k_max=32) for _ in range(3)]
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


@pytest.mark.parametrize("k_max", [1, 32])
def test_full_size_overdetermined(L, ctx, k_max):
    """4096 x 2048 dense U[0,1) problem with noise, as benchmarked."""
    A, b, _ = WL.overdetermined_uniform(0)
    x, P, _, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max)
    assert_parity(x, P, info, ref, counters=False)


def test_full_size_sparse_recovery(L, ctx):
    """2048 x 8192 unit-column Gaussian, s = 128, noiseless: exact recovery,
    checked against the known x0 and the KKT conditions (any size)."""
    A, b, x0 = WL.sparse_recovery_sweep(0, 128)
    x, P, _, info = solve(L, ctx, A, b, k_max=64)
    assert info["status"] == 0
    assert P.tolist() == np.flatnonzero(x0).tolist()
    assert np.linalg.norm(x - x0) <= RTOL * np.linalg.norm(x0)
