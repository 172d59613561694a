"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each check uses an independent
source - hand-derived fixtures, brute-force enumeration with numpy's least
squares, scipy's nnls, closed forms, theorems of the paper, or a fresh QR.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_05345_gb300 import workloads as WL

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def kkt_residuals(A, b, x, passive):
    """Theorem 1 (KKT, section 2): returns (min x_P, max |x_Z|, max w_Z, max |w_P|)."""
    w = A.T @ (b - A @ x)
    n = A.shape[1]
    P = np.zeros(n, dtype=bool)
    P[list(passive)] = True
    return (x[P].min() if P.any() else np.inf, np.abs(x[~P]).max() if (~P).any() else 0.0,
            w[~P].max() if (~P).any() else -np.inf, np.abs(w[P]).max() if P.any() else 0.0)


def assert_kkt(A, b, r, scale=None):
    x = r["x"]
    xmin, xz, wz, wp = kkt_residuals(A, b, x, r["passive"])
    tol = r["tol_w"] * 10 if scale is None else scale
    assert xmin > 0.0
    assert xz == 0.0
    assert wz <= tol, (wz, tol)
    assert wp <= tol, (wp, tol)


# ---------------------------------------------------------------- hand-derived
@pytest.mark.parametrize("k_max", [1, 4])
def test_golden_small_nnls(k_max):
    data = json.load(open(os.path.join(GOLD, "nnls_small.json")))
    for case in data["cases"]:
        A = np.array(case["A_rows"], dtype=float)
        b = np.array(case["b"], dtype=float)
        r = O.nnls(A, b, k_max=k_max)
        assert r["status"] == O.OK
        np.testing.assert_allclose(r["x"], case["x"], rtol=0, atol=1e-14, err_msg=case["name"])
        assert r["passive"].tolist() == case["passive"], case["name"]
        assert abs(r["resid_norm"] - case["resid"]) <= 1e-14 * max(1.0, case["resid"])


def test_golden_dm_cases():
    data = json.load(open(os.path.join(GOLD, "dm_cases.json")))
    base = data["base"]
    C = np.array(base["C_columns"], dtype=float).T
    # the prescribed pairwise cosines hold by construction
    Cn = C / np.linalg.norm(C, axis=0)
    assert abs(Cn[:, 0] @ Cn[:, 1] - 0.5) < 1e-15 and abs(Cn[:, 0] @ Cn[:, 2] - 0.95) < 1e-15
    for case in data["cases"]:
        w = np.array(case.get("w", base["w"]))
        u = np.array(case.get("u", base["u"]))
        J = O.dm_select(C, w, u, case["tau1"], case["tau2"], case["delta"], case["k_max"])
        assert J == case["J"], (case["name"], J, case["why"])


# ---------------------------------------------------------------- brute force
def brute_force_nnls(A, b):
    """Enumerate every support S (|S| <= rank): least squares on S; keep the
    feasible ones (y >= 0); the smallest residual is the NNLS optimum."""
    m, n = A.shape
    best = (np.linalg.norm(b), np.zeros(n), ())
    for k in range(1, min(m, n) + 1):
        for S in itertools.combinations(range(n), k):
            AS = A[:, S]
            y, *_ = np.linalg.lstsq(AS, b, rcond=None)
            if np.all(y >= 0):
                res = np.linalg.norm(AS @ y - b)
                if res < best[0] - 1e-13:
                    x = np.zeros(n)
                    x[list(S)] = y
                    best = (res, x, S)
    return best


@pytest.mark.parametrize("shape", [(8, 12), (12, 8)])
@pytest.mark.parametrize("k_max", [1, 4])
def test_brute_force_enumeration(shape, k_max):
    m, n = shape
    for seed in range(40):
        A, b = WL.tiny(seed, m, n)
        res_bf, x_bf, S_bf = brute_force_nnls(A, b)
        r = O.nnls(A, b, k_max=k_max)
        assert r["status"] == O.OK
        assert abs(r["resid_norm"] - res_bf) <= 1e-10 * max(1.0, np.linalg.norm(b)), (seed, r["resid_norm"], res_bf)
        if m >= n:  # full column rank: strictly convex, the minimiser is unique
            np.testing.assert_allclose(r["x"], x_bf, atol=1e-10 * max(1.0, np.abs(x_bf).max()))
            assert set(r["passive"].tolist()) == set(np.flatnonzero(x_bf > 0).tolist())
        assert_kkt(A, b, r, scale=1e-9)


# ---------------------------------------------------------------- library pin
def test_scipy_nnls_agreement():
    scipy_opt = pytest.importorskip("scipy.optimize")
    for seed in range(4):
        A, b, _ = WL.overdetermined_uniform(seed, m=384, n=192)
        xs, rs = scipy_opt.nnls(A, b, maxiter=50 * 192)
        for k in (1, 16):
            r = O.nnls(A, b, k_max=k)
            assert r["status"] == O.OK
            np.testing.assert_allclose(r["x"], xs, rtol=0, atol=1e-9 * np.abs(xs).max())
            assert set(r["passive"].tolist()) == set(np.flatnonzero(xs > 0).tolist())
            assert abs(r["resid_norm"] - rs) <= 1e-10 * rs


# ---------------------------------------------------------------- closed forms
def test_single_column_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.normal(size=(7, 1))
        b = rng.normal(size=7)
        r = O.nnls(a, b, k_max=1)
        expect = max(float(a[:, 0] @ b), 0.0) / float(a[:, 0] @ a[:, 0])
        assert abs(r["x"][0] - expect) <= 1e-15 * max(1.0, expect)


def test_orthonormal_columns_closed_form():
    rng = np.random.default_rng(4)
    for k in (1, 8):
        Q, _ = np.linalg.qr(rng.normal(size=(50, 20)))
        b = rng.normal(size=50)
        r = O.nnls(Q, b, k_max=k)
        np.testing.assert_allclose(r["x"], np.maximum(Q.T @ b, 0.0), atol=1e-14)


def test_positive_least_squares_is_nnls():
    rng = np.random.default_rng(5)
    A = rng.uniform(0.5, 1.5, size=(60, 10)) + np.eye(60, 10) * 3
    y = rng.uniform(1.0, 2.0, size=10)
    b = A @ y + 1e-3 * rng.normal(size=60)
    ls = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.all(ls > 0)
    for k in (1, 4, 10):
        r = O.nnls(A, b, k_max=k)
        np.testing.assert_allclose(r["x"], ls, rtol=1e-12, atol=0)
        assert r["n_passive"] == 10


def test_empty_and_degenerate_problems():
    r = O.nnls(np.zeros((5, 0)), np.ones(5))
    assert r["status"] == O.OK and r["n_passive"] == 0
    r = O.nnls(np.zeros((4, 3)), np.ones(4), k_max=2)
    assert r["status"] == O.OK and r["n_passive"] == 0 and not r["x"].any()
    r = O.nnls(np.ones((4, 3)), np.zeros(4), k_max=2)
    assert r["status"] == O.OK and not r["x"].any()


def test_status_codes():
    A, b, _ = WL.small_recovery(0)
    A2 = A.copy()
    A2[3, 7] = np.nan
    assert O.nnls(A2, b)["status"] == O.NONFINITE
    b2 = b.copy()
    b2[0] = np.inf
    assert O.nnls(A, b2)["status"] == O.NONFINITE
    assert O.nnls(A, b, k_max=1, max_outer=3)["status"] == O.MAX_ITER


# ---------------------------------------------------------------- paper's claims
@pytest.mark.parametrize("k_max", [1, 8])
def test_exact_recovery_small(k_max):
    """Noiseless sparse nonnegative recovery (section 3; the paper reports exact
    recovery on all ERC instances, section 5)."""
    for seed in range(8):
        A, b, x0 = WL.small_recovery(seed)
        r = O.nnls(A, b, k_max=k_max, trace=True)
        assert r["status"] == O.OK
        assert r["passive"].tolist() == np.flatnonzero(x0).tolist()
        assert np.linalg.norm(r["x"] - x0) <= 1e-10 * np.linalg.norm(x0)
        assert_kkt(A, b, r)


@pytest.mark.parametrize("k_max", [1, 8, 32])
def test_strict_decrease_and_kkt_with_noise(k_max):
    """Theorem 3 (section 2.2): the objective strictly decreases at every outer
    step, so the passive sets never repeat; on exit KKT holds."""
    for seed in range(3):
        A, b, _ = WL.overdetermined_uniform(seed, m=320, n=160)
        r = O.nnls(A, b, k_max=k_max, trace=True)
        assert r["status"] == O.OK
        res = r["trace_resid"]
        assert np.all(np.diff(res) < 0)
        assert_kkt(A, b, r)


def test_no_feasibility_drops_when_tau1_is_one():
    """Theorem 4: with tau1 = 1 and tau2 <= 1/2, y_J > 0 at every outer step,
    so the feasibility loop never drops a column."""
    for seed in range(6):
        for A, b in [WL.small_recovery(seed)[:2], WL.overdetermined_uniform(seed, m=300, n=150)[:2]]:
            r = O.nnls(A, b, k_max=8, tau1=1.0, tau2=0.5, trace=True)
            assert r["status"] == O.OK
            assert r["n_drop"] == 0


def test_lh_and_lhdm_agree():
    """Both algorithms stop at the KKT point (Theorems 1 and 3), unique here."""
    for seed in range(4):
        A, b, _ = WL.overdetermined_uniform(seed, m=400, n=200)
        r1 = O.nnls(A, b, k_max=1)
        for k in (8, 32):
            rk = O.nnls(A, b, k_max=k)
            assert rk["passive"].tolist() == r1["passive"].tolist()
            assert np.linalg.norm(rk["x"] - r1["x"]) <= 1e-11 * np.linalg.norm(r1["x"])
            assert rk["n_outer"] < r1["n_outer"]


def test_lhdm_takes_blocks():
    A, b, x0 = WL.small_recovery(1)
    r = O.nnls(A, b, k_max=8, trace=True)
    assert r["trace"][:, 1].max() > 1  # DM appended several columns at once
    assert r["trace"][0, 0] >= r["trace"][0, 1] >= 1


# ---------------------------------------------------------------- QR modification
def _abs_rows_equal(R1, R2, tol):
    return np.max(np.abs(np.abs(R1) - np.abs(R2))) <= tol


def test_updating_matches_fresh_qr():
    """Algorithm 4 reproduces the R of a fresh QR of the appended columns, up to
    row signs, and keeps Q^T b consistent with the least-squares residual."""
    rng = np.random.default_rng(11)
    A = rng.normal(size=(40, 25))
    b = rng.normal(size=40)
    st = O.QRState(A, b)
    assert st.append([3, 7, 1]) == 3
    assert st.append([20, 4]) == 2
    s = st.get()
    order = s["order"].tolist()
    assert order == [3, 7, 1, 20, 4]
    Rf = np.linalg.qr(A[:, order], mode="r")
    assert _abs_rows_equal(s["R"], Rf, 1e-12 * np.abs(Rf).max())
    # orthogonal transforms keep column norms of the whole matrix and of b
    np.testing.assert_allclose(np.linalg.norm(s["W"], axis=0), np.linalg.norm(A, axis=0), rtol=1e-13)
    assert abs(np.linalg.norm(s["bt"]) - np.linalg.norm(b)) <= 1e-13 * np.linalg.norm(b)
    # residual identity: ||b - A_P y|| = ||(Q^T b)_{nP+1:m}||
    y = np.linalg.lstsq(A[:, order], b, rcond=None)[0]
    assert abs(np.linalg.norm(b - A[:, order] @ y) - np.linalg.norm(s["bt"][5:])) <= 1e-12


def test_drop_last_restores_state():
    rng = np.random.default_rng(12)
    A = rng.normal(size=(30, 12))
    b = rng.normal(size=30)
    s1 = O.QRState(A, b)
    s1.append([2, 5, 9])
    s1.drop_last()
    s2 = O.QRState(A, b)
    s2.append([2, 5])
    g1, g2 = s1.get(), s2.get()
    assert g1["order"].tolist() == g2["order"].tolist() == [2, 5]
    np.testing.assert_allclose(g1["W"], g2["W"], atol=1e-13)
    np.testing.assert_allclose(g1["bt"], g2["bt"], atol=1e-13)


@pytest.mark.parametrize("positions", [[0], [3], [1, 4], [0, 2, 5], [6]])
def test_downdating_matches_fresh_qr(positions):
    """Algorithm 5 gives the R of a fresh QR of the remaining columns (same
    order), up to row signs, and keeps W = Q^T A orthogonally equivalent."""
    rng = np.random.default_rng(13)
    A = rng.normal(size=(35, 20))
    b = rng.normal(size=35)
    st = O.QRState(A, b)
    cols = [5, 1, 17, 8, 0, 12, 3]
    st.append(cols)
    assert st.delete(positions) == 0
    s = st.get()
    keep = [c for p, c in enumerate(cols) if p not in positions]
    assert s["order"].tolist() == keep
    Rf = np.linalg.qr(A[:, keep], mode="r")
    assert _abs_rows_equal(s["R"], Rf, 1e-12 * np.abs(Rf).max())
    np.testing.assert_allclose(np.linalg.norm(s["W"], axis=0), np.linalg.norm(A, axis=0), rtol=1e-13)
    k = len(keep)
    y = np.linalg.lstsq(A[:, keep], b, rcond=None)[0]
    assert abs(np.linalg.norm(b - A[:, keep] @ y) - np.linalg.norm(s["bt"][k:])) <= 1e-12
    # the removed columns are back in trailing form: their C norms equal the
    # norms of their projections off span(A_P)
    Qk, _ = np.linalg.qr(A[:, keep])
    for p in positions:
        c = cols[p]
        proj = A[:, c] - Qk @ (Qk.T @ A[:, c])
        assert abs(np.linalg.norm(s["W"][k:, c]) - np.linalg.norm(proj)) <= 1e-12


def test_final_R_matches_fresh_qr_after_solve():
    A, b, _ = WL.overdetermined_uniform(2, m=300, n=150)
    r = O.nnls(A, b, k_max=8, want_R=True, trace=True)
    assert r["n_inner"] > 0  # the solve went through downdates
    Rf = np.linalg.qr(A[:, r["order"]], mode="r")
    assert _abs_rows_equal(r["R"], Rf, 1e-11 * np.abs(Rf).max())


# ---------------------------------------------------------------- adjoint
def test_adjoint_closed_form_vs_finite_differences():
    """dL/db and dL/dA_P of the dense closed form against central differences
    (h = 1e-6) of the oracle's own solve, on a stable passive set."""
    from oracle.adjoint import nnls_adjoint
    rng = np.random.default_rng(21)
    m, n = 40, 60
    A = rng.normal(0, 1 / np.sqrt(m), size=(m, n))
    x0 = np.zeros(n)
    x0[rng.choice(n, 6, replace=False)] = rng.uniform(0.5, 1.0, 6)
    b = A @ x0 + 1e-3 * rng.normal(size=m)
    xt = x0 + 1e-2 * rng.normal(size=n)
    base = O.nnls(A, b, k_max=8)
    P = base["passive"].tolist()
    g = 2 * (base["x"] - xt)
    dLdb, dLdA = nnls_adjoint(A, b, base["x"], P, g)
    h = 1e-6

    def loss(Ax, bx):
        r = O.nnls(Ax, bx, k_max=8)
        assert r["passive"].tolist() == P
        return float(np.sum((r["x"] - xt) ** 2))

    fd_b = np.array([(loss(A, b + h * e) - loss(A, b - h * e)) / (2 * h) for e in np.eye(m)[:10]])
    np.testing.assert_allclose(fd_b, dLdb[:10], rtol=1e-5, atol=1e-7)
    for (i, j) in [(0, P[0]), (5, P[1]), (17, P[-1]), (3, P[2])]:
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (loss(A + E, b) - loss(A - E, b)) / (2 * h)
        assert abs(fd - dLdA[i, j]) <= 1e-5 * max(1.0, abs(fd)), (i, j, fd, dLdA[i, j])
    Z = [j for j in range(n) if j not in P]
    assert not dLdA[:, Z].any()


# ---------------------------------------------------------------- rank guard
@pytest.mark.parametrize("seed", range(4))
def test_rank_guard_truncates_dependent_block(seed):
    """A DM block {a6, a1, a4} with a6 = a1 + a4 (a1, a4 orthonormal; pairwise
    cosines 1/sqrt(2) and 0, all below delta = 0.9, so Algorithm 2 accepts all
    three).  With b = 1.2 a1 + a4 = a6 + 0.2 a1: w = A^T b gives w6 = 2.2 (the
    argmax), w1 = 1.2, w4 = 1.0, so with tau1 = 0.4 both are candidates, in
    that order.  After the reflectors of a6 and a1 the trailing part of a4 is
    at the rounding level: the rank guard (a column whose trailing norm is
    <= 100 eps ||a_j|| cannot enter) ends J there, so two columns are
    appended, y = (1, 0.2) > 0 (no drop), the residual is zero and the solve
    stops after one outer step with x6 = 1, x1 = 0.2.  Appending the third
    column (the guard skipped) puts a rounding-level pivot into R and moves
    the solution to another point of the optimal set."""
    A, b, (i1, i2, i3) = WL.dependent_triple(seed=seed)
    w = A.T @ b
    assert np.argmax(w) == i3 and sorted(np.argsort(-w)[:3].tolist()) == sorted([i1, i2, i3])
    r = O.nnls(A, b, k_max=8, tau1=0.4, trace=True)
    assert r["status"] == O.OK
    assert r["trace"][0].tolist() == [3, 2, 0, 2, 0, i3]
    assert r["n_drop"] == 0
    assert r["n_outer"] == 1 and r["passive"].tolist() == sorted([i1, i3])
    expect = np.zeros(A.shape[1])
    expect[i3], expect[i1] = 1.0, 0.2
    np.testing.assert_allclose(r["x"], expect, rtol=0, atol=1e-14)
    # the optimum value is zero (b lies in the cone of the columns)
    assert r["resid_norm"] <= 1e-14
    res_bf, _, _ = brute_force_nnls(A, b)
    assert res_bf <= 1e-14


@pytest.mark.parametrize("k_max", [1, 4])
@pytest.mark.parametrize("where", ["after", "before"])
def test_duplicate_column_takes_lowest_index(k_max, where):
    """An exact copy of a passive column: the two copies tie in every
    comparison (w and the trailing norm), the argmax tie rule picks the
    lower index, and once it is passive the copy's trailing part is zero, so
    it never enters.  The solution is the one of the original matrix with
    the coefficient on the lower-indexed copy, the optimum value unchanged
    (brute force agrees)."""
    for seed in range(6):
        A, b = WL.tiny(seed, 12, 8)
        base = O.nnls(A, b, k_max=k_max)
        P = base["passive"].tolist()
        c = P[0]
        at = A.shape[1] if where == "after" else c  # copy after all, or just before c
        A2 = WL.with_duplicate(A, c, at)
        r = O.nnls(A2, b, k_max=k_max)
        assert r["status"] == O.OK
        x_expect = np.insert(base["x"], at, 0.0)
        if where == "before":  # the copy now has the lower index: it carries the coefficient
            x_expect[at], x_expect[c + 1] = base["x"][c], 0.0
        np.testing.assert_allclose(r["x"], x_expect, rtol=0, atol=1e-12 * max(1.0, np.abs(base["x"]).max()))
        both = {at, c if where == "after" else c + 1}
        assert not both <= set(r["passive"].tolist())
        assert abs(r["resid_norm"] - base["resid_norm"]) <= 1e-12 * max(1.0, np.linalg.norm(b))


# ---------------------------------------------------------------- conditioned workload
@pytest.mark.parametrize("kappa", [1e5, 1e6])
def test_conditioned_problem_matches_scipy(kappa):
    """Ill-conditioned overdetermined NNLS (condition numbers 1e5 - 1e6 as in
    the paper's conditioned experiment): the minimiser is unique (full column
    rank), so the oracle and scipy's independent active-set solver must agree
    to the conditioning-limited accuracy, with the same support."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    A, b, _ = WL.conditioned_overdetermined(0, m=512, n=256, kappa=kappa)
    assert 0.3 * kappa < np.linalg.cond(A) < 3 * kappa
    xs, _ = scipy_opt.nnls(A, b, maxiter=50 * 256)
    for k in (1, 16):
        r = O.nnls(A, b, k_max=k)
        assert r["status"] == O.OK
        assert np.linalg.norm(r["x"] - xs) <= 1e-10 * np.linalg.norm(xs)
        assert set(r["passive"].tolist()) == set(np.flatnonzero(xs > 0).tolist())
        assert_kkt(A, b, r)


@pytest.mark.parametrize("kappa", [1e5, 1e6])
def test_conditioned_sparse_recovery(kappa):
    """Noiseless sparse nonnegative recovery with an ill-conditioned A: x0 is
    recovered (the paper reports LHDM solving every such instance)."""
    for s in (16, 32):
        A, b, x0 = WL.conditioned_recovery(0, s=s, kappa=kappa)
        r = O.nnls(A, b, k_max=32)
        assert r["status"] == O.OK
        assert np.linalg.norm(r["x"] - x0) <= 1e-10 * np.linalg.norm(x0)
        sig = np.flatnonzero(r["x"] > 1e-9 * r["x"].max()).tolist()
        assert sig == np.flatnonzero(x0).tolist()


# ---------------------------------------------------------------- positivity trick
@pytest.mark.parametrize("flip", [False, True])
@pytest.mark.parametrize("k_max", [1, 8])
def test_positivity_trick_is_least_squares(flip, k_max):
    """Section 3.2: NNLS on [A -A] reaches every signed vector, so for a full
    column rank A (m > n) its optimum is the least-squares solution:
    x+ - x- = lstsq(A, b) and the optimal residuals agree.  The twin rule
    keeps at most one column of each pair passive (x+ * x- = 0)."""
    for seed in range(3):
        A, b, _ = WL.signed_overdetermined(seed, m=120, n=60)
        r = O.nnls_signed(A, b, sign_flip=flip, k_max=k_max)
        assert r["status"] == O.OK
        n = A.shape[1]
        xp, xm = r["x"][:n], r["x"][n:]
        ls = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.linalg.norm((xp - xm) - ls) <= 1e-11 * np.linalg.norm(ls)
        assert not (xp * xm).any()
        assert xp.min() >= 0 and xm.min() >= 0
        assert abs(r["resid_norm"] - np.linalg.norm(A @ ls - b)) <= 1e-12 * np.linalg.norm(b)
        if flip:
            assert r["n_flip"] > 0 or r["n_inner"] == 0


def test_sign_flip_replaces_inner_loop():
    """Section 4.2: with the positivity trick the sign flip takes the place of
    the inner loop's downdates (each flip keeps y up to one sign), so on the
    same instance the flip variant runs no (or fewer) inner steps, flips
    instead, and reaches the same optimum."""
    A, b, _ = WL.signed_overdetermined(1, m=200, n=100)
    r_in = O.nnls_signed(A, b, sign_flip=False, k_max=1)
    r_fl = O.nnls_signed(A, b, sign_flip=True, k_max=1)
    assert r_in["n_inner"] > 0 and r_in["n_flip"] == 0
    assert r_fl["n_flip"] > 0 and r_fl["n_inner"] < r_in["n_inner"]
    n = A.shape[1]
    d_in = r_in["x"][:n] - r_in["x"][n:]
    d_fl = r_fl["x"][:n] - r_fl["x"][n:]
    assert np.linalg.norm(d_in - d_fl) <= 1e-11 * np.linalg.norm(d_in)


@pytest.mark.parametrize("flip", [False, True])
def test_positivity_trick_signed_recovery(flip):
    """Noiseless signed sparse recovery: x+ = max(x0, 0), x- = max(-x0, 0)."""
    for seed in range(4):
        A, b, x0 = WL.signed_recovery(seed)
        r = O.nnls_signed(A, b, sign_flip=flip, k_max=8)
        n = A.shape[1]
        expect = np.concatenate([np.maximum(x0, 0), np.maximum(-x0, 0)])
        assert r["status"] == O.OK
        assert np.linalg.norm(r["x"] - expect) <= 1e-10 * np.linalg.norm(expect)
        # at a zero residual, columns with rounding-level coefficients may
        # stay passive: the significant part is the support of x0
        sig = np.flatnonzero(r["x"] > 1e-9 * r["x"].max()).tolist()
        assert sig == np.flatnonzero(expect).tolist()
        assert set(sig) <= set(r["passive"].tolist())


def test_positivity_trick_brute_force():
    """Tiny underdetermined cases (m = 6, n = 4, so [A -A] is 6 x 8): the
    oracle's optimum equals brute-force enumeration on the explicit [A -A]."""
    for seed in range(10):
        A, b = WL.tiny(seed, 6, 4)
        A2 = np.hstack([A, -A])
        res_bf, _, _ = brute_force_nnls(A2, b)
        for flip in (False, True):
            r = O.nnls_signed(A, b, sign_flip=flip, k_max=4)
            assert abs(r["resid_norm"] - res_bf) <= 1e-10 * max(1.0, np.linalg.norm(b))


# ---------------------------------------------------------------- l1-NNLS
def l1_subgradient_gap(A, b, lam, xs):
    """Optimality of x = x+ - x- for f(x) = ||x||_1^2 + lam^2 ||A x - b||^2
    (the objective of eq. (l1_NNLS) once x+ * x- = 0): with
    g = lam^2 A^T (b - A x) and t = ||x||_1, 0 is in the subdifferential
    iff g_i = t sign(x_i) where x_i != 0 and |g_i| <= t where x_i = 0.
    Returns the largest violation relative to t."""
    g = lam * lam * (A.T @ (b - A @ xs))
    t = np.abs(xs).sum()
    nz = xs != 0
    v1 = np.abs(g[nz] - t * np.sign(xs[nz])).max() if nz.any() else 0.0
    v2 = max(0.0, (np.abs(g[~nz]) - t).max()) if (~nz).any() else 0.0
    return max(v1, v2) / max(t, 1e-300)


@pytest.mark.parametrize("lam", [0.5, 3.0, 30.0])
def test_l1_nnls_optimality(lam):
    """The oracle's l1-NNLS solution, with x = x+ - x-, minimises
    ||x||_1^2 + lam^2 ||A x - b||^2: the subgradient condition holds, the two
    halves never overlap, and the stacked residual equals the objective."""
    for seed in range(3):
        A, b, _ = WL.signed_recovery(seed, m=60, n=120, s=8)
        for k in (1, 8):
            r = O.nnls_l1(A, b, lam, k_max=k)
            assert r["status"] == O.OK
            n = A.shape[1]
            xp, xm = r["x"][:n], r["x"][n:]
            assert not (xp * xm).any()
            xs = xp - xm
            assert l1_subgradient_gap(A, b, lam, xs) <= 1e-9
            f = np.abs(xs).sum() ** 2 + lam * lam * np.sum((A @ xs - b) ** 2)
            assert abs(r["resid_norm"] ** 2 - f) <= 1e-10 * max(1.0, f)


def test_l1_nnls_single_column_closed_form():
    """n = 1: min x^2 + lam^2 ||a x - b||^2 gives x = lam^2 a^T b / (1 + lam^2 ||a||^2)."""
    rng = np.random.default_rng(8)
    for _ in range(10):
        a = rng.normal(size=(9, 1))
        b = rng.normal(size=9)
        lam = rng.uniform(0.2, 5.0)
        r = O.nnls_l1(a, b, lam, k_max=2)
        xs = r["x"][0] - r["x"][1]
        expect = lam ** 2 * float(a[:, 0] @ b) / (1.0 + lam ** 2 * float(a[:, 0] @ a[:, 0]))
        assert abs(xs - expect) <= 1e-14 * max(1.0, abs(expect))


def test_l1_nnls_brute_force():
    """Tiny cases: the oracle's optimum equals brute-force enumeration on the
    explicit stacked matrix (5 x 8)."""
    for seed in range(8):
        A, b = WL.tiny(seed, 4, 4)
        M, rhs = O.l1_stack(A, b, 2.0)
        res_bf, _, _ = brute_force_nnls(M, rhs)
        r = O.nnls_l1(A, b, 2.0, k_max=4)
        assert abs(r["resid_norm"] - res_bf) <= 1e-10 * max(1.0, np.linalg.norm(rhs))
