"""The tensor-core commit (exact 7-bit digit products on bf16 tensor cores
for the block reflector update, 5 <= k <= 32) against the oracle on inputs
built to strain it, and its accuracy guard's FP64 fallbacks:

- rows of A scaled by powers of two over 2^-15 .. 2^15 (so the columns of
  C' = 2^Er C, whose digits pass 1 multiplies, span 2^-30 .. 2^30), at
  k_max 12 and 32 (also with columns scaled over 2^-2 .. 2^2);
- a nearly dependent pair of columns inside the DM block;
- the guard's fallback forced on (every batch to FP64): the result must not
  move beyond rounding.
Bar: identical passive set, trace and counters, ||x - x_oracle|| <= 1e-10
||x_oracle||."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2108_05345_gb300 import workloads as WL
from gpu_util import RTOL, assert_parity, solve

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
    c = L.Context(1024, 1024)
    yield c
    c.close()


def scaled(seed, rr, cc, m=700, n=350):
    A, b, _ = WL.overdetermined_uniform(seed, m=m, n=n)
    rng = np.random.default_rng(11 + seed)
    rs = 2.0 ** rng.integers(-rr, rr + 1, size=m)
    cs = 2.0 ** rng.integers(-cc, cc + 1, size=n)
    return np.asfortranarray(A * rs[:, None] * cs[None, :]), b * rs


@pytest.mark.parametrize("rr,cc", [(15, 0), (12, 0), (15, 2)])
@pytest.mark.parametrize("k_max", [12, 32])
def test_wide_scales(L, ctx, rr, cc, k_max):
    A, b = scaled(5, rr, cc)
    x, P, _, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max, trace=True)
    assert ref["status"] == 0 and max(ref["trace"][:, 1]) >= 5  # the tensor-core commit ran
    assert_parity(x, P, info, ref, trace=ctx.trace())


def test_nearly_dependent_block(L, ctx):
    A, b, _ = WL.overdetermined_uniform(6, m=600, n=300)
    rng = np.random.default_rng(2)
    # pairs of columns at cosine ~ 0.89 (accepted by delta = 0.9 together)
    for j in range(0, 40, 2):
        A[:, j + 1] = A[:, j] + 0.52 * np.linalg.norm(A[:, j]) / np.sqrt(600) * rng.standard_normal(600)
    A = np.asfortranarray(A)
    x, P, _, info = solve(L, ctx, A, b, k_max=32)
    ref = O.nnls(A, b, k_max=32, trace=True)
    assert_parity(x, P, info, ref, trace=ctx.trace())


@pytest.mark.parametrize("mode", [1])
def test_forced_fallbacks(L, ctx, mode):
    A, b = scaled(7, 12, 0)
    ref = O.nnls(A, b, k_max=24, trace=True)
    ctx.force_commit_guard(mode)
    try:
        x, P, _, info = solve(L, ctx, A, b, k_max=24)
        ctl = ctx.state("ctl", 16)
    finally:
        ctx.force_commit_guard(0)
    assert ctl[10] > 0  # the fallback ran
    assert_parity(x, P, info, ref, trace=ctx.trace())
