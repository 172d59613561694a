"""ctypes front end of the C oracle (test infrastructure only).

Every array crosses the boundary as contiguous FP64 / int32 numpy memory;
A is passed column-major (Fortran order).  See lhdm_oracle.c for what each
entry point computes and the paper passages it follows.
"""
import ctypes as C
import numpy as np

from .build_oracle import build

_lib = None

OK, INVALID_ARG, MAX_ITER, NONFINITE = 0, 1, 2, 4


class _Params(C.Structure):
    _fields_ = [("tau1", C.c_double), ("tau2", C.c_double), ("delta", C.c_double),
                ("k_max", C.c_int), ("tol_w", C.c_double), ("max_outer", C.c_int),
                ("twin_n", C.c_int), ("sign_flip", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("n_outer", C.c_int), ("n_inner", C.c_int),
                ("n_drop", C.c_int), ("n_passive", C.c_int), ("rank_limited", C.c_int),
                ("n_flip", C.c_int),
                ("resid_norm", C.c_double), ("max_wZ", C.c_double), ("tol_w", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i = C.POINTER(C.c_double), C.POINTER(C.c_int)
        _lib.orc_nnls.argtypes = [C.c_int, C.c_int, d, C.c_int, d, C.POINTER(_Params), d, i,
                                  C.POINTER(_Info), C.c_int, i, d, d]
        _lib.orc_nnls.restype = C.c_int
        _lib.orc_dm_select.argtypes = [C.c_int, C.c_int, d, C.c_int, d, d, C.c_double,
                                       C.c_double, C.c_double, C.c_int, i]
        _lib.orc_dm_select.restype = C.c_int
        _lib.orc_state_new.argtypes = [C.c_int, C.c_int, d, C.c_int, d, C.c_int]
        _lib.orc_state_new.restype = C.c_void_p
        _lib.orc_state_free.argtypes = [C.c_void_p]
        _lib.orc_state_append.argtypes = [C.c_void_p, C.c_int, i]
        _lib.orc_state_append.restype = C.c_int
        _lib.orc_state_drop_last.argtypes = [C.c_void_p]
        _lib.orc_state_delete.argtypes = [C.c_void_p, C.c_int, i]
        _lib.orc_state_delete.restype = C.c_int
        _lib.orc_state_get.argtypes = [C.c_void_p, i, i, d, d, d]
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def nnls(A, b, k_max=1, tau1=0.6, tau2=0.15, delta=0.9, tol_w=-1.0, max_outer=0,
         trace=False, want_R=False, twin_n=0, sign_flip=False):
    """Solve min ||Ax-b|| s.t. x >= 0 by LH (k_max=1) or LHDM (k_max>1).

    Returns a dict: x, order (ordered passive set), passive (sorted), info
    fields, and optionally trace (rows: |J| from DM, |J| kept, inner steps,
    nP after, removed, first column j) with the per-step residual norms and
    decision margins, and R.
    """
    A = np.asfortranarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m, n = A.shape
    x = np.zeros(n)
    order = np.full(n, -1, dtype=np.int32)
    prm = _Params(tau1, tau2, delta, int(k_max), tol_w, int(max_outer), int(twin_n), int(bool(sign_flip)))
    inf = _Info()
    cap = 4 * n + 8 if trace else 0
    ti = np.zeros(6 * max(cap, 1), dtype=np.int32)
    td = np.zeros(2 * max(cap, 1))
    R = np.zeros(min(m, n) ** 2) if want_R else None
    lib().orc_nnls(m, n, _dp(A), m, _dp(b), C.byref(prm), _dp(x), _ip(order), C.byref(inf),
                   cap, _ip(ti) if trace else None, _dp(td) if trace else None,
                   _dp(R) if want_R else None)
    nP = inf.n_passive
    out = dict(x=x, order=order[:nP].copy(), passive=np.sort(order[:nP]), status=inf.status,
               n_outer=inf.n_outer, n_inner=inf.n_inner, n_drop=inf.n_drop, n_passive=nP,
               rank_limited=inf.rank_limited, resid_norm=inf.resid_norm, max_wZ=inf.max_wZ,
               tol_w=inf.tol_w, n_flip=inf.n_flip)
    if trace:
        no = min(inf.n_outer, cap)
        out["trace"] = ti[: 6 * no].reshape(no, 6).copy()
        out["trace_resid"] = td[0:2 * no:2].copy()
        out["trace_margin"] = td[1:2 * no:2].copy()
    if want_R:
        out["R"] = R[: nP * nP].reshape(nP, nP, order="F").copy()
    return out


def nnls_signed(A, b, sign_flip=False, **kw):
    """Signed least squares through the positivity trick (section 3.2): NNLS
    on the explicit matrix [A  -A], x = (x+, x-) of length 2n; with
    sign_flip, the inner loop's downdate for a negative y is replaced by the
    sign flip of section 4.2.  Returns the dict of nnls()."""
    A = np.asarray(A, dtype=np.float64)
    A2 = np.asfortranarray(np.hstack([A, -A]))
    return nnls(A2, b, twin_n=A.shape[1], sign_flip=sign_flip, **kw)


def l1_stack(A, b, lam):
    """The l1-NNLS system of section 3.3, eq. (l1_NNLS), written out: the
    (m+1) x 2n matrix [1^T 1^T; lam A  -lam A] and the right-hand side
    [0; lam b] (column-major)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    M = np.empty((m + 1, 2 * n))
    M[0, :] = 1.0
    M[1:, :n] = lam * A
    M[1:, n:] = -lam * A
    rhs = np.concatenate([[0.0], lam * np.asarray(b, dtype=np.float64)])
    return np.asfortranarray(M), rhs


def nnls_l1(A, b, lam, **kw):
    """l1-NNLS (section 3.3): NNLS on l1_stack(A, b, lam); x = (x+, x-) of
    length 2n.  Returns the dict of nnls()."""
    M, rhs = l1_stack(A, b, lam)
    return nnls(M, rhs, **kw)


def dm_select(C_, w, u, tau1, tau2, delta, k_max):
    """Algorithm 2 on an explicit candidate matrix; returns the ordered J."""
    C_ = np.asfortranarray(C_, dtype=np.float64)
    L, nc = C_.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    J = np.full(max(k_max, 1), -1, dtype=np.int32)
    k = lib().orc_dm_select(L, nc, _dp(C_), L, _dp(w), _dp(u), tau1, tau2, delta, int(k_max), _ip(J))
    return J[:k].tolist()


class QRState:
    """The oracle's whole-matrix partial QR state Q^T [A | b] (Algorithms 4, 5)."""

    def __init__(self, A, b, kcap=64):
        self.A = np.asfortranarray(A, dtype=np.float64)
        self.b = np.ascontiguousarray(b, dtype=np.float64)
        self.m, self.n = self.A.shape
        self.h = lib().orc_state_new(self.m, self.n, _dp(self.A), self.m, _dp(self.b), kcap)
        if not self.h:
            raise ValueError("bad shape")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_state_free(self.h)
            self.h = None

    def append(self, cols):
        c = np.ascontiguousarray(cols, dtype=np.int32)
        return lib().orc_state_append(self.h, len(c), _ip(c))

    def drop_last(self):
        lib().orc_state_drop_last(self.h)

    def delete(self, positions):
        q = np.ascontiguousarray(sorted(positions), dtype=np.int32)
        return lib().orc_state_delete(self.h, len(q), _ip(q))

    def get(self):
        nP = C.c_int(0)
        lib().orc_state_get(self.h, C.byref(nP), None, None, None, None)
        k = nP.value
        order = np.zeros(max(k, 1), dtype=np.int32)
        R = np.zeros(max(k * k, 1))
        bt = np.zeros(self.m)
        W = np.zeros(self.m * self.n)
        lib().orc_state_get(self.h, C.byref(nP), _ip(order), _dp(R), _dp(bt), _dp(W))
        return dict(nP=k, order=order[:k].copy(), R=R[: k * k].reshape(k, k, order="F").copy(),
                    bt=bt, W=W.reshape(self.m, self.n, order="F"))
