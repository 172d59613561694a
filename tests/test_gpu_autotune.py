"""Autotuner of the batched solve: the table it fills, the k_max a batch then
takes per instance, and the solutions at those k_max against the CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
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
    yield lhdm
    lhdm.tuning_set([0] * lhdm.TUNE_BUCKETS)


def to_dev(L, A, b):
    At = L.colmajor(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    return At, torch.from_numpy(np.ascontiguousarray(b)).cuda()


def test_autotune_table_and_use(L):
    L.tuning_set([0] * L.TUNE_BUCKETS)
    inst = [(A, b) for A, b, _ in WL.batched_uneven(batch_seed=7, count=18, m_lo=40, m_hi=200)]
    dev = [to_dev(L, A, b) for A, b in inst]
    As, bs = [d[0] for d in dev], [d[1] for d in dev]
    table = L.batch_autotune(As, bs, L.default_params())
    present = {L.tune_bucket(A.shape[1]) for A, _ in inst}
    for bkt in range(L.TUNE_BUCKETS):
        if bkt in present:
            assert table[bkt] in L.TUNE_CANDIDATES
        else:
            assert table[bkt] == 0
    assert L.tuning_get() == table
    batch = L.Batch(As, bs, L.default_params(k_max=0))
    batch.run()
    torch.cuda.synchronize()
    infos = batch.info()
    for i, (A, b) in enumerate(inst):
        k = batch.kmax(i)
        assert k == table[L.tune_bucket(A.shape[1])]
        ref = O.nnls(A, b, k_max=k, trace=True)
        x = batch.xs[i].cpu().numpy()
        p = batch.ps[i].cpu().numpy()
        assert infos[i]["status"] == ref["status"] == 0
        tied = (ref["trace_margin"] < TIE).any() if len(ref["trace_margin"]) else False
        if not tied:
            assert p[p >= 0].tolist() == ref["passive"].tolist()
        assert np.linalg.norm(x - ref["x"]) <= RTOL * max(np.linalg.norm(ref["x"]), 1e-300)
    batch.close()


def test_tuning_set_get_and_errors(L):
    L.tuning_set([4, 8, 16, 32, 32, 0])
    assert L.tuning_get() == [4, 8, 16, 32, 32, 0]
    with pytest.raises(RuntimeError):
        L.tuning_set([4, 8, 16, 32, 65, 0])
    assert L.tuning_get() == [4, 8, 16, 32, 32, 0]
    L.tuning_set([0] * L.TUNE_BUCKETS)
    assert L.tuning_get() == [0] * L.TUNE_BUCKETS
