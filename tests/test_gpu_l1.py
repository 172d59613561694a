"""l1-NNLS (section 3.3, eq. (l1_NNLS)) on the GPU against the CPU oracle.

lhdm_solve_l1 builds the stacked (m+1) x 2n system [1^T 1^T; lam A -lam A],
(0; lam b) with a kernel and solves it; the oracle solves the same system
written out in numpy.  Bar: identical sorted passive set of the stacked
system, ||x - x_oracle|| <= 1e-10 ||x_oracle||, identical counters and
decision trace, over a sweep of lam."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2108_05345_gb300 import workloads as WL
from gpu_util import assert_parity, dev

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
    c = L.Context(1025, 4096)
    yield c
    c.close()


def check(L, ctx, A, b, lam, k_max):
    At, bt = dev(L, A, b)
    x, p, info = ctx.solve_l1(At, bt, lam, L.default_params(k_max=k_max))
    ref = O.nnls_l1(A, b, lam, k_max=k_max, trace=True)
    ps = p.cpu().numpy()
    assert_parity(x.cpu().numpy(), ps[ps >= 0], info, ref, trace=ctx.trace())
    assert len(ps) == 2 * A.shape[1]
    return x.cpu().numpy()


@pytest.mark.parametrize("lam", [0.5, 3.0, 30.0])
@pytest.mark.parametrize("k_max", [1, 8])
def test_l1_small(L, ctx, lam, k_max):
    for seed in range(3):
        A, b, _ = WL.signed_recovery(seed, m=60, n=120, s=8)
        check(L, ctx, A, b, lam, k_max)


@pytest.mark.parametrize("lam", [1.0, 10.0, 100.0])
def test_l1_sweep_larger(L, ctx, lam):
    """A 512 x 1024 (the stacked system is 513 x 2048), noisy signed sparse
    data; larger lam weighs the residual more and the solution approaches the
    sparse x0."""
    A, b0, x0 = WL.signed_recovery(0, m=512, n=1024, s=40)
    b = b0 + 1e-3 * np.random.default_rng(5).normal(size=512)
    x = check(L, ctx, A, b, lam, 32)
    n = A.shape[1]
    xs = x[:n] - x[n:]
    if lam >= 100.0:
        assert np.linalg.norm(xs - x0) <= 0.05 * np.linalg.norm(x0)


def test_l1_refuses_bad_arguments(L, ctx):
    A, b, _ = WL.signed_recovery(0, m=60, n=120, s=8)
    At, bt = dev(L, A, b)
    with pytest.raises(RuntimeError):
        ctx.solve_l1(At, bt, -1.0)
    with pytest.raises(RuntimeError):
        ctx.solve_l1(At, bt, 1.0, L.default_params(mode=1))
