"""Helpers shared by the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import torch

RTOL = 1e-10
# A decision whose comparison is this close to flipping (relative) is taken
# by rounding; from that step on only the final result is compared.
TIE = 1e-9


def dev(L, A, b):
    At = L.colmajor(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    return At, torch.from_numpy(np.ascontiguousarray(b)).cuda()


def solve(L, ctx, A, b, **kw):
    At, bt = dev(L, A, b)
    x, p, info = ctx.solve(At, bt, L.default_params(**kw))
    torch.cuda.synchronize()
    ps = p.cpu().numpy()
    return x.cpu().numpy(), ps[ps >= 0], ps, info


def first_divergence(tr_gpu, tr_ref, margin):
    for s in range(min(len(tr_gpu), len(tr_ref))):
        if margin[s] < TIE:
            return None
        if not np.array_equal(tr_gpu[s], tr_ref[s]):
            return s, tr_gpu[s].tolist(), tr_ref[s].tolist()
    if len(tr_gpu) != len(tr_ref):
        return len(tr_ref), None, None
    return None


def significant(v):
    return np.flatnonzero(v > 1e-9 * max(np.abs(v).max(), 1e-300)).tolist()


def assert_parity(x, P, info, ref, counters=True, trace=None):
    """Identical sorted passive set, ||x - x_oracle|| <= 1e-10 ||x_oracle||,
    same status and counters; a rounding tie in the oracle's path relaxes the
    passive-set check to the significant support."""
    assert info["status"] == ref["status"], (info, ref["status"])
    tied = "trace_margin" in ref and len(ref["trace_margin"]) and (ref["trace_margin"] < TIE).any()
    if counters and trace is not None and "trace" in ref:
        d = first_divergence(trace, ref["trace"], ref["trace_margin"])
        assert d is None, "decision trace diverges at outer step %s: gpu %s oracle %s" % d
    counters = counters and not tied
    if tied:
        assert significant(x) == significant(ref["x"])
    else:
        assert P.tolist() == ref["passive"].tolist()
    nx = max(np.linalg.norm(ref["x"]), 1e-300)
    assert np.linalg.norm(x - ref["x"]) <= RTOL * nx or (np.linalg.norm(ref["x"]) == 0 and not x.any())
    if counters:
        assert (info["n_outer"], info["n_inner"], info["n_drop"]) == (ref["n_outer"], ref["n_inner"], ref["n_drop"])
    assert abs(info["resid_norm"] - ref["resid_norm"]) <= 1e-9 * max(1.0, ref["resid_norm"])


def kkt(A, b, x, tol_w):
    """(min over x >= 0 violations, max w over the zero set, |w| on the support)."""
    w = A.T @ (b - A @ x)
    Z = x == 0
    return (x.min(), w[Z].max() if Z.any() else -np.inf, np.abs(w[~Z]).max() if (~Z).any() else 0.0)
