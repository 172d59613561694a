"""CUDA path vs the CPU oracle on the ill-conditioned workload (condition
numbers 1e5 and 1e6, the range of the paper's conditioned experiment):

- dense overdetermined NNLS with a unique minimiser, A 2048 x 1024: identical
  passive set, decision trace and counters, ||x - x_oracle|| <= 1e-10
  ||x_oracle||, for LH and LHDM;
- noiseless sparse recovery, A 512 x 1024: x0 recovered to 1e-10 and the
  oracle's x matched to 1e-10 (these instances reach a zero residual, where
  decisions on rounding-level coefficients are ties, so the passive set is
  compared on its significant part)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2108_05345_gb300 import workloads as WL
from gpu_util import RTOL, assert_parity, significant, solve

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
    c = L.Context(2048, 1024)
    yield c
    c.close()


@pytest.mark.parametrize("kappa", [1e5, 1e6])
@pytest.mark.parametrize("k_max", [1, 32])
def test_conditioned_overdetermined(L, ctx, kappa, k_max):
    A, b, _ = WL.conditioned_overdetermined(0, kappa=kappa)
    x, P, _, info = solve(L, ctx, A, b, k_max=k_max)
    ref = O.nnls(A, b, k_max=k_max, trace=True)
    assert ref["n_inner"] > 0
    assert_parity(x, P, info, ref, trace=ctx.trace())


@pytest.mark.parametrize("kappa", [1e5, 1e6])
@pytest.mark.parametrize("s", [16, 64])
def test_conditioned_recovery(L, ctx, kappa, s):
    A, b, x0 = WL.conditioned_recovery(0, s=s, kappa=kappa)
    x, P, _, info = solve(L, ctx, A, b, k_max=32)
    ref = O.nnls(A, b, k_max=32)
    assert info["status"] == 0
    assert np.linalg.norm(x - x0) <= RTOL * np.linalg.norm(x0)
    assert np.linalg.norm(x - ref["x"]) <= RTOL * np.linalg.norm(ref["x"])
    assert significant(x) == significant(ref["x"]) == np.flatnonzero(x0).tolist()
