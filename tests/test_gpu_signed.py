"""Positivity trick (section 3.2: NNLS on [A -A], signed solutions) and the
sign flip of section 4.2, CUDA path vs the CPU oracle.

The CUDA path never forms -A: it keeps a sign per passive column.  The
oracle solves NNLS on the explicit [A -A] (oracle.nnls_signed).  Bar: the
identical sorted passive set of [A -A] indices, ||x - x_oracle|| <= 1e-10
||x_oracle|| on the 2n-vector (x+, x-), identical status, outer, inner,
drop and flip counts and decision trace."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2108_05345_gb300 import workloads as WL
from gpu_util import RTOL, assert_parity, dev, significant

pytestmark = pytest.mark.gpu
MODES = {"inner": 1, "flip": 2}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05345_gb300 import build, lhdm
    build.build()
    return lhdm


@pytest.fixture(scope="module")
def ctx(L):
    c = L.Context(2048, 8192)
    yield c
    c.close()


def solve_signed(L, ctx, A, b, mode, **kw):
    At, bt = dev(L, A, b)
    x, p, info = ctx.solve(At, bt, L.default_params(mode=mode, **kw))
    torch.cuda.synchronize()
    ps = p.cpu().numpy()
    return x.cpu().numpy(), ps[ps >= 0], ps, info


@pytest.mark.parametrize("variant", ["inner", "flip"])
@pytest.mark.parametrize("k_max", [1, 32])
@pytest.mark.parametrize("seed", range(3))
def test_signed_least_squares(L, ctx, variant, k_max, seed):
    A, b, _ = WL.signed_overdetermined(seed)
    x, P, ps, info = solve_signed(L, ctx, A, b, MODES[variant], k_max=k_max)
    ref = O.nnls_signed(A, b, sign_flip=variant == "flip", k_max=k_max, trace=True)
    assert_parity(x, P, info, ref, trace=ctx.trace())
    assert info["n_flip"] == ref["n_flip"] and info["mode"] == MODES[variant]
    assert (ps[len(P):] == -1).all() and len(ps) == 2 * A.shape[1]
    n = A.shape[1]
    assert not (x[:n] * x[n:]).any()


@pytest.mark.parametrize("variant", ["inner", "flip"])
def test_signed_recovery_small(L, ctx, variant):
    for seed in range(4):
        A, b, x0 = WL.signed_recovery(seed)
        x, P, _, info = solve_signed(L, ctx, A, b, MODES[variant], k_max=8)
        ref = O.nnls_signed(A, b, sign_flip=variant == "flip", k_max=8, trace=True)
        assert_parity(x, P, info, ref, trace=ctx.trace())
        expect = np.concatenate([np.maximum(x0, 0), np.maximum(-x0, 0)])
        assert np.linalg.norm(x - expect) <= RTOL * np.linalg.norm(expect)


@pytest.mark.parametrize("variant", ["inner", "flip"])
def test_signed_recovery_sparse_recovery_size(L, ctx, variant):
    """2048 x 8192 unit-norm Gaussian columns (the sparse-recovery sweep's
    matrix), signed x0 with 128 nonzeros: [A -A] is 2048 x 16384."""
    A, b, x0 = WL.signed_recovery(0, m=2048, n=8192, s=128, unit_columns=True)
    x, P, _, info = solve_signed(L, ctx, A, b, MODES[variant], k_max=64)
    ref = O.nnls_signed(A, b, sign_flip=variant == "flip", k_max=64)
    expect = np.concatenate([np.maximum(x0, 0), np.maximum(-x0, 0)])
    assert info["status"] == 0
    assert np.linalg.norm(x - expect) <= RTOL * np.linalg.norm(expect)
    assert np.linalg.norm(x - ref["x"]) <= RTOL * np.linalg.norm(ref["x"])
    assert significant(x) == np.flatnonzero(expect).tolist()


@pytest.mark.parametrize("variant", ["inner", "flip"])
def test_signed_batched(L, variant):
    inst = [WL.signed_overdetermined(s, m=150 + 37 * s, n=70 + 11 * s) for s in range(6)]
    dv = [dev(L, A, b) for A, b, _ in inst]
    prm = L.default_params(mode=MODES[variant], k_max=8)
    batch = L.Batch([d[0] for d in dv], [d[1] for d in dv], prm)
    batch.run()
    torch.cuda.synchronize()
    infos = batch.info()
    for i, (A, b, _) in enumerate(inst):
        ref = O.nnls_signed(A, b, sign_flip=variant == "flip", k_max=8, trace=True)
        p = batch.ps[i].cpu().numpy()
        assert_parity(batch.xs[i].cpu().numpy(), p[p >= 0], infos[i], ref)
        assert infos[i]["n_flip"] == ref["n_flip"]
    batch.close()


def test_signed_mode_has_no_adjoint(L, ctx):
    A, b, _ = WL.signed_overdetermined(0, m=60, n=30)
    At, bt = dev(L, A, b)
    ctx.solve(At, bt, L.default_params(mode=1, k_max=4))
    with pytest.raises(RuntimeError):
        ctx.backward(At, torch.zeros(60, dtype=torch.float64, device="cuda"))
