"""The allocation-free entry point (lhdm_solve_noalloc) against lhdm_solve.

lhdm_solve_noalloc is for callers that may not allocate device memory; it
runs the same kernel on a fixed workspace compiled into the library.  This
test calls it through the C ABI twice in a row (a maximum-size instance,
then a smaller ragged one, so the second call starts from the first call's
leftovers in the shared workspace) and checks each result against the
context-based lhdm_solve: identical sorted passive set, identical counters,
||x - x_ref|| <= 1e-10 ||x_ref||.  It also checks that an oversized problem
is refused before anything is launched.  Kept in its own file, collected
last, so a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest
import torch

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


def test_noalloc_matches_context_solve_twice(L):
    cases = [WL.small_recovery(3)[:2], WL.tiny(77, 131, 257)]
    ctx = L.Context(256, 512)
    prm = L.default_params(k_max=8)
    for A, b in cases:
        At = L.colmajor(torch.from_numpy(np.ascontiguousarray(A)).cuda())
        bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        x_ref, p_ref, info_ref = ctx.solve(At, bt, prm)
        rc, x, p, info = L.solve_noalloc(At, bt, prm)
        assert rc == L.LHDM_OK, L.status_string(rc)
        torch.cuda.synchronize()
        inf = L.info_from_device(info)
        xr = x_ref.cpu().numpy()
        assert p.cpu().numpy().tolist() == p_ref.cpu().numpy().tolist()
        assert np.linalg.norm(x.cpu().numpy() - xr) <= RTOL * np.linalg.norm(xr)
        for k in ("status", "n_outer", "n_inner", "n_drop", "n_passive"):
            assert inf[k] == info_ref[k], k
    ctx.close()


def test_noalloc_refuses_oversized_problem(L):
    A = L.colmajor(torch.zeros(257, 4, dtype=torch.float64, device="cuda"))
    b = torch.zeros(257, dtype=torch.float64, device="cuda")
    rc, *_ = L.solve_noalloc(A, b)
    assert rc == L.LHDM_ERR_TOO_LARGE
    A = L.colmajor(torch.zeros(4, 513, dtype=torch.float64, device="cuda"))
    b = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc, *_ = L.solve_noalloc(A, b)
    assert rc == L.LHDM_ERR_TOO_LARGE
