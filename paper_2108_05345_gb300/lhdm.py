"""Python binding of liblhdm.so (include/lhdm.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels; PyTorch supplies
device memory and streams.  The library must have been built (build.py);
importing this module on a machine without it raises instead of falling
back to anything else.

Matrices are column-major FP64: pass A as a (m, n) torch tensor with
stride (1, lda), e.g. ``colmajor(A)``.
"""
import ctypes as C
import os

import torch

from . import build as _build

LHDM_OK = 0
LHDM_ERR_INVALID_ARG = 1
LHDM_ERR_MAX_ITER = 2
LHDM_ERR_NONFINITE = 4
LHDM_ERR_CUDA = 5
LHDM_ERR_TIMEOUT = 6
LHDM_ERR_ALLOC = 7
LHDM_ERR_NO_STATE = 8
LHDM_ERR_TOO_LARGE = 9
KMAX_LIMIT = 64
MODE_NNLS, MODE_SIGNED, MODE_SIGNED_FLIP = 0, 1, 2
PHASES = ("setup", "dm", "panel", "solve", "commit", "inner", "residual", "dual",
          "feasibility", "chain", "zrot", "inner_trsv")


class Params(C.Structure):
    _fields_ = [("tau1", C.c_double), ("tau2", C.c_double), ("delta", C.c_double),
                ("tol_w", C.c_double), ("k_max", C.c_int32), ("max_outer", C.c_int32),
                ("mode", C.c_int32), ("reserved", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_outer", C.c_int32), ("n_inner", C.c_int32),
                ("n_drop", C.c_int32), ("n_passive", C.c_int32), ("rank_limited", C.c_int32),
                ("n_flip", C.c_int32), ("mode", C.c_int32),
                ("resid_norm", C.c_double), ("max_wZ", C.c_double), ("tol_w", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Loads liblhdm.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("liblhdm.so is not built; run paper_2108_05345_gb300/build.py "
                               "(or __graft_entry__.build()) on a machine with nvcc")
        L = C.CDLL(_build.LIB)
        P, I, V = C.POINTER(Params), C.POINTER(Info), C.c_void_p
        d, i32 = C.c_void_p, C.c_int32
        L.lhdm_default_params.argtypes = [P]
        L.lhdm_status_string.argtypes = [C.c_int]
        L.lhdm_status_string.restype = C.c_char_p
        L.lhdm_create.argtypes = [C.POINTER(V), i32, i32, i32]
        L.lhdm_destroy.argtypes = [V]
        L.lhdm_solve.argtypes = [V, i32, i32, d, i32, d, P, d, d, I, V]
        L.lhdm_solve_host.argtypes = [V, i32, i32, d, i32, d, P, d, d, I, V]
        L.lhdm_solve_noalloc.argtypes = [i32, i32, d, i32, d, P, d, d, d, V]
        L.lhdm_get_info.argtypes = [V, I, V]
        L.lhdm_backward.argtypes = [V, i32, d, i32, d, d, d, i32, V]
        L.lhdm_set_wait_limit.argtypes = [V, C.c_int64]
        L.lhdm_solve_l1.argtypes = [V, i32, i32, d, i32, d, C.c_double, P, d, d, I, V]
        L.lhdm_debug_stall_next_solve.argtypes = [V]
        L.lhdm_debug_commit_guard.argtypes = [V, i32]
        L.lhdm_debug_fast_math.argtypes = [V, V, i32, V]
        L.lhdm_phase_times.argtypes = [V, C.POINTER(C.c_double), i32, V]
        L.lhdm_trace.argtypes = [V, C.POINTER(C.c_int32), i32, V]
        L.lhdm_debug_state.argtypes = [V, C.c_char_p, C.c_void_p, C.c_int64, V]
        pp = C.POINTER(C.c_void_p)
        ip = C.POINTER(C.c_int32)
        L.lhdm_batch_create.argtypes = [C.POINTER(V), i32, ip, ip, ip, pp, pp, pp, pp, d, P, V]
        L.lhdm_batch_run.argtypes = [V, V]
        L.lhdm_batch_backward.argtypes = [V, pp, pp, pp, ip, V]
        L.lhdm_solve_batched.argtypes = [V, i32, ip, ip, pp, ip, pp, P, pp, pp, d, V]
        L.lhdm_backward_batched.argtypes = [V, pp, pp, pp, ip, V]
        L.lhdm_batch_kmax.argtypes = [V, i32]
        L.lhdm_batch_destroy.argtypes = [V]
        L.lhdm_batch_autotune.argtypes = [i32, ip, ip, ip, pp, pp, P, ip, V]
        L.lhdm_tuning_get.argtypes = [ip]
        L.lhdm_tuning_set.argtypes = [ip]
        _lib = L
    return _lib


def status_string(s):
    return lib().lhdm_status_string(int(s)).decode()


def _check(rc, what):
    if rc != LHDM_OK:
        raise RuntimeError("%s failed: %s (%d)" % (what, status_string(rc), rc))


def default_params(**kw):
    p = Params()
    lib().lhdm_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def colmajor(A):
    """(m, n) tensor -> the same values with column-major strides (1, m)."""
    return A.t().contiguous().t()


def _lda(A):
    m, n = A.shape
    if A.dtype != torch.float64:
        raise TypeError("A must be float64")
    if m == 0 or n == 0:
        return max(1, m)  # no element is read
    if n == 1 and A.stride(0) == 1:
        return max(1, m)
    if m == 1 and A.stride(1) >= 1:
        return A.stride(1)  # a single row: the column stride is the leading dimension
    if A.stride(0) != 1 or A.stride(1) < max(1, m):
        raise ValueError("A must be column-major (stride (1, lda >= m)); use colmajor(A)")
    return A.stride(1)


def _nx(n, params):
    """Length of x and of the passive list: n, or 2n in the signed modes."""
    return 2 * n if (params is not None and params.mode != MODE_NNLS) else n


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def solve_noalloc(A, b, params=None, x=None, passive=None, info=None, stream=None):
    """lhdm_solve_noalloc: the solve without any device allocation inside
    the library (fixed static workspace; m <= 256, n <= 512).  x, passive
    and info (a device buffer of one lhdm_info, as 6 float64) may be given
    by the caller; returns the raw status code and the three tensors."""
    m, n = A.shape
    lda = _lda(A)
    dev = A.device
    nx = _nx(n, params)
    if x is None:
        x = torch.empty(nx, dtype=torch.float64, device=dev)
    if passive is None:
        passive = torch.empty(nx, dtype=torch.int32, device=dev)
    if info is None:
        info = torch.zeros(C.sizeof(Info) // 8, dtype=torch.float64, device=dev)
    rc = lib().lhdm_solve_noalloc(m, n, A.data_ptr() if A.numel() else None, lda,
                                  b.data_ptr() if b.numel() else None,
                                  C.byref(params) if params is not None else None,
                                  x.data_ptr() if n else None, passive.data_ptr() if n else None,
                                  info.data_ptr(), _stream(stream))
    return rc, x, passive, info


def fast_math(x, stream=None):
    """lhdm_debug_fast_math on a CUDA float64 tensor x: an (n, 4) tensor of
    (solver 1/x, 1.0/x, solver sqrt|x|, sqrt|x|)."""
    import torch
    x = x.contiguous()
    out = torch.empty((x.numel(), 4), dtype=torch.float64, device=x.device)
    _check(lib().lhdm_debug_fast_math(x.data_ptr(), out.data_ptr(), x.numel(), _stream(stream)),
           "lhdm_debug_fast_math")
    return out


def info_from_device(buf):
    """An lhdm_info held in a device float64 buffer -> dict."""
    return Info.from_buffer_copy(buf.cpu().numpy().tobytes()).as_dict()


def _ptrs(ts):
    return (C.c_void_p * max(len(ts), 1))(*[t.data_ptr() if t is not None else None for t in ts])


def _ints(vals):
    return (C.c_int32 * max(len(vals), 1))(*vals)


class Context:
    """A solve context (lhdm_create) for single problems up to max_m x max_n
    and batches of up to max_batch such problems."""

    def __init__(self, max_m, max_n, max_batch=0):
        h = C.c_void_p()
        _check(lib().lhdm_create(C.byref(h), int(max_m), int(max_n), int(max_batch)), "lhdm_create")
        self.h = h
        self.max_m, self.max_n, self.max_batch = int(max_m), int(max_n), int(max_batch)
        self._batch_keep = None

    def close(self):
        if getattr(self, "h", None):
            lib().lhdm_destroy(self.h)
            self.h = None

    __del__ = close

    def solve(self, A, b, params=None, x=None, passive=None, stream=None, sync=True):
        """lhdm_solve on device tensors; returns (x, passive, info dict or None)."""
        m, n = A.shape
        lda = _lda(A)
        if b.dtype != torch.float64 or b.numel() != m or not b.is_contiguous():
            raise ValueError("b must be a contiguous float64 vector of length m")
        nx = _nx(n, params)
        if x is None:
            x = torch.empty(nx, dtype=torch.float64, device=A.device)
        if passive is None:
            passive = torch.empty(nx, dtype=torch.int32, device=A.device)
        if x.numel() < nx or passive.numel() < nx:
            raise ValueError("x and passive need %d entries" % nx)
        info = Info() if sync else None
        rc = lib().lhdm_solve(self.h, m, n, A.data_ptr(), lda, b.data_ptr(),
                              C.byref(params) if params is not None else None,
                              x.data_ptr(), passive.data_ptr(),
                              C.byref(info) if info is not None else None, _stream(stream))
        _check(rc, "lhdm_solve")
        return x, passive, (info.as_dict() if info is not None else None)

    def solve_batched(self, As, bs, params=None, xs=None, ps=None, infos=None, stream=None):
        """lhdm_solve_batched: one persistent launch over the instances (lists
        of column-major (m_i, n_i) tensors and length-m_i vectors).  Returns
        (xs, passives, infos) with infos a device float64 buffer of the
        per-instance lhdm_info records (info_list() decodes it).  Passing the
        same tensors again reuses the context's plan (capturable)."""
        k = len(As)
        dev = As[0].device if k else torch.device("cuda")
        if xs is None:
            xs = [torch.empty(_nx(A.shape[1], params), dtype=torch.float64, device=dev) for A in As]
        if ps is None:
            ps = [torch.empty(_nx(A.shape[1], params), dtype=torch.int32, device=dev) for A in As]
        if infos is None:
            infos = torch.zeros(max(k, 1) * C.sizeof(Info) // 8, dtype=torch.float64, device=dev)
        m = _ints([A.shape[0] for A in As])
        n = _ints([A.shape[1] for A in As])
        lda = _ints([_lda(A) for A in As])
        for b, A in zip(bs, As):
            if b.dtype != torch.float64 or b.numel() != A.shape[0] or not b.is_contiguous():
                raise ValueError("every b must be a contiguous float64 vector of its A's row count")
        rc = lib().lhdm_solve_batched(self.h, k, m, n, _ptrs(As), lda, _ptrs(bs),
                                      C.byref(params) if params is not None else None,
                                      _ptrs(xs), _ptrs(ps), infos.data_ptr(), _stream(stream))
        _check(rc, "lhdm_solve_batched")
        self._batch_keep = (As, bs, xs, ps, infos)
        return xs, ps, infos

    @staticmethod
    def info_list(infos, count):
        raw = infos.cpu().numpy().tobytes()
        sz = C.sizeof(Info)
        return [Info.from_buffer_copy(raw[i * sz:(i + 1) * sz]).as_dict() for i in range(count)]

    def backward_batched(self, As, dLdx, want_db=True, want_dA=True, stream=None):
        """lhdm_backward_batched for the last solve_batched; returns lists
        (dL/db, dL/dA) (column-major dL/dA)."""
        dbs = [torch.empty(A.shape[0], dtype=torch.float64, device=A.device) for A in As] if want_db else None
        dAs = [colmajor(torch.empty(A.shape, dtype=torch.float64, device=A.device)) for A in As] if want_dA else None
        gs = [g.contiguous() if g is not None else None for g in dLdx]
        ld = _ints([max(1, A.shape[0]) for A in As])
        rc = lib().lhdm_backward_batched(self.h, _ptrs(gs), _ptrs(dbs) if dbs else None,
                                         _ptrs(dAs) if dAs else None, ld, _stream(stream))
        _check(rc, "lhdm_backward_batched")
        return dbs, dAs

    def solve_host(self, A, b, params=None, stream=None):
        """lhdm_solve_host on host arrays (numpy, Fortran order or any layout
        with unit row stride); returns (x, passive, info dict)."""
        import numpy as np
        A = np.asfortranarray(A, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        m, n = A.shape
        x = np.empty(_nx(n, params), dtype=np.float64)
        p = np.empty(_nx(n, params), dtype=np.int32)
        info = Info()
        rc = lib().lhdm_solve_host(self.h, m, n, A.ctypes.data, max(1, m), b.ctypes.data,
                                   C.byref(params) if params is not None else None,
                                   x.ctypes.data, p.ctypes.data, C.byref(info), _stream(stream))
        _check(rc, "lhdm_solve_host")
        return x, p, info.as_dict()

    def solve_host_ptr(self, m, n, A_ptr, lda, b_ptr, x_ptr, p_ptr, params=None, stream=None):
        """lhdm_solve_host on raw host pointers (e.g. pinned torch tensors)."""
        info = Info()
        rc = lib().lhdm_solve_host(self.h, m, n, A_ptr, lda, b_ptr,
                                   C.byref(params) if params is not None else None,
                                   x_ptr, p_ptr, C.byref(info), _stream(stream))
        _check(rc, "lhdm_solve_host")
        return info.as_dict()

    def info(self, stream=None):
        inf = Info()
        _check(lib().lhdm_get_info(self.h, C.byref(inf), _stream(stream)), "lhdm_get_info")
        return inf.as_dict()

    def backward(self, A, dLdx, want_db=True, want_dA=True, idx=-1, stream=None):
        """lhdm_backward: adjoint of the last solve (idx < 0) or of instance
        idx of the last solve_batched; returns (dL/db, dL/dA)."""
        m, n = A.shape
        lda = _lda(A)
        db = torch.empty(m, dtype=torch.float64, device=A.device) if want_db else None
        dA = colmajor(torch.empty(m, n, dtype=torch.float64, device=A.device)) if want_dA else None
        rc = lib().lhdm_backward(self.h, int(idx), A.data_ptr(), lda, dLdx.contiguous().data_ptr(),
                                 db.data_ptr() if db is not None else None,
                                 dA.data_ptr() if dA is not None else None, max(1, m), _stream(stream))
        _check(rc, "lhdm_backward")
        return db, dA

    def solve_l1(self, A, b, lam, params=None, x=None, passive=None, stream=None, sync=True):
        """lhdm_solve_l1: l1-NNLS (section 3.3) with weight lam; returns
        (x of length 2n = (x+, x-), passive of the stacked system, info)."""
        m, n = A.shape
        lda = _lda(A)
        if b.dtype != torch.float64 or b.numel() != m or not b.is_contiguous():
            raise ValueError("b must be a contiguous float64 vector of length m")
        if x is None:
            x = torch.empty(2 * n, dtype=torch.float64, device=A.device)
        if passive is None:
            passive = torch.empty(2 * n, dtype=torch.int32, device=A.device)
        info = Info() if sync else None
        rc = lib().lhdm_solve_l1(self.h, m, n, A.data_ptr(), lda, b.data_ptr(), float(lam),
                                 C.byref(params) if params is not None else None,
                                 x.data_ptr(), passive.data_ptr(),
                                 C.byref(info) if info is not None else None, _stream(stream))
        _check(rc, "lhdm_solve_l1")
        return x, passive, (info.as_dict() if info is not None else None)

    def l1_path(self, A, b, lams, params=None):
        """l1-NNLS for each weight of a sweep; returns a list of (x, passive, info)."""
        return [tuple(t.clone() if torch.is_tensor(t) else t for t in self.solve_l1(A, b, lam, params))
                for lam in lams]

    def set_wait_limit(self, ns):
        _check(lib().lhdm_set_wait_limit(self.h, int(ns)), "lhdm_set_wait_limit")

    def force_commit_guard(self, mode):
        _check(lib().lhdm_debug_commit_guard(self.h, int(mode)), "lhdm_debug_commit_guard")

    def stall_next_solve(self):
        _check(lib().lhdm_debug_stall_next_solve(self.h), "lhdm_debug_stall_next_solve")

    def trace(self, stream=None):
        """Per outer step: |J| from DM, |J| kept, inner steps, |P| after,
        removed, first column of J (lhdm_trace)."""
        import numpy as np
        cap = 3 * self.max_n + 8
        buf = (C.c_int32 * (6 * cap))()
        k = lib().lhdm_trace(self.h, buf, cap, _stream(stream))
        if k < 0:
            raise RuntimeError("lhdm_trace failed")
        return np.frombuffer(buf, dtype=np.int32)[: 6 * k].reshape(k, 6).copy()

    def state(self, name, count, stream=None):
        """lhdm_debug_state: a named piece of the solver state as numpy."""
        import numpy as np
        dt = np.int32 if name in ("order", "rslot", "pos", "ctl") else np.float64
        out = np.empty(int(count), dtype=dt)
        _check(lib().lhdm_debug_state(self.h, name.encode(), out.ctypes.data, int(count), _stream(stream)),
               "lhdm_debug_state")
        return out

    def phase_times(self, stream=None):
        """{phase: ms} of the last solve (lhdm_phase_times)."""
        return self.profile(stream)[0]

    def profile(self, stream=None):
        """({phase: ms}, {phase: algorithmic FP64 flops}) of the last solve."""
        ms, fl, _ = self.profile_full(stream)
        return ms, fl

    def profile_full(self, stream=None):
        """({phase: ms}, {phase: algorithmic FP64 flops}, bf16 MMA
        instructions of the tensor-core commit) of the last solve."""
        n = 2 * len(PHASES) + 1
        buf = (C.c_double * n)()
        k = lib().lhdm_phase_times(self.h, buf, n, _stream(stream))
        if k < n:
            raise RuntimeError("lhdm_phase_times failed")
        ms = {PHASES[i]: buf[i] for i in range(len(PHASES))}
        fl = {PHASES[i]: buf[len(PHASES) + i] for i in range(len(PHASES))}
        return ms, fl, buf[2 * len(PHASES)]


class Batch:
    """A planned batch of independent solves (lhdm_batch_create); run() is
    one persistent launch and may be captured in a CUDA graph."""

    def __init__(self, As, bs, params=None, stream=None):
        self.As = As
        self.bs = bs
        k = len(As)
        self.k = k
        dev = As[0].device if k else torch.device("cuda")
        self.xs = [torch.empty(_nx(A.shape[1], params), dtype=torch.float64, device=dev) for A in As]
        self.ps = [torch.empty(_nx(A.shape[1], params), dtype=torch.int32, device=dev) for A in As]
        self.infos = torch.zeros(max(k, 1) * C.sizeof(Info) // 8, dtype=torch.float64, device=dev)
        m = (C.c_int32 * max(k, 1))(*[A.shape[0] for A in As])
        n = (C.c_int32 * max(k, 1))(*[A.shape[1] for A in As])
        lda = (C.c_int32 * max(k, 1))(*[_lda(A) for A in As])
        ptrs = lambda ts: (C.c_void_p * max(k, 1))(*[t.data_ptr() for t in ts])
        self._keep = (m, n, lda)
        h = C.c_void_p()
        rc = lib().lhdm_batch_create(C.byref(h), k, m, n, lda, ptrs(As), ptrs(bs), ptrs(self.xs),
                                     ptrs(self.ps), self.infos.data_ptr(),
                                     C.byref(params) if params is not None else None, _stream(stream))
        _check(rc, "lhdm_batch_create")
        self.h = h

    def run(self, stream=None):
        _check(lib().lhdm_batch_run(self.h, _stream(stream)), "lhdm_batch_run")

    def info(self):
        raw = self.infos.cpu().numpy().tobytes()
        out = []
        for i in range(self.k):
            inf = Info.from_buffer_copy(raw[i * C.sizeof(Info):(i + 1) * C.sizeof(Info)])
            out.append(inf.as_dict())
        return out

    def kmax(self, i):
        return lib().lhdm_batch_kmax(self.h, i)

    def backward(self, dLdx, want_db=True, want_dA=True, stream=None):
        k = self.k
        dbs = [torch.empty(A.shape[0], dtype=torch.float64, device=A.device) for A in self.As] if want_db else None
        dAs = [colmajor(torch.empty(A.shape, dtype=torch.float64, device=A.device)) for A in self.As] if want_dA else None
        ptrs = lambda ts: (C.c_void_p * max(k, 1))(*[t.data_ptr() for t in ts])
        ld = (C.c_int32 * max(k, 1))(*[max(1, A.shape[0]) for A in self.As])
        gs = [g.contiguous() for g in dLdx]  # kept alive across the call
        rc = lib().lhdm_batch_backward(self.h, ptrs(gs),
                                       ptrs(dbs) if dbs else None, ptrs(dAs) if dAs else None, ld,
                                       _stream(stream))
        _check(rc, "lhdm_batch_backward")
        return dbs, dAs

    def close(self):
        if getattr(self, "h", None):
            lib().lhdm_batch_destroy(self.h)
            self.h = None

    __del__ = close


TUNE_BUCKETS = 6  # LHDM_TUNE_BUCKETS
TUNE_CANDIDATES = (4, 8, 16, 32)


def tune_bucket(n):
    """Size bucket of the autotuner for an instance with n columns."""
    b, lim = 0, 128
    while b < TUNE_BUCKETS - 1 and n > lim:
        b, lim = b + 1, lim * 2
    return b


def batch_autotune(As, bs, params=None, stream=None):
    """Times every candidate k_max per size bucket on these instances
    (lhdm_batch_autotune) and returns the tuner's table (list of ints)."""
    k = len(As)
    m = (C.c_int32 * max(k, 1))(*[A.shape[0] for A in As])
    n = (C.c_int32 * max(k, 1))(*[A.shape[1] for A in As])
    lda = (C.c_int32 * max(k, 1))(*[_lda(A) for A in As])
    ptrs = lambda ts: (C.c_void_p * max(k, 1))(*[t.data_ptr() for t in ts])
    table = (C.c_int32 * TUNE_BUCKETS)()
    rc = lib().lhdm_batch_autotune(k, m, n, lda, ptrs(As), ptrs(bs),
                                   C.byref(params) if params is not None else None, table, _stream(stream))
    _check(rc, "lhdm_batch_autotune")
    return list(table)


def tuning_get():
    table = (C.c_int32 * TUNE_BUCKETS)()
    _check(lib().lhdm_tuning_get(table), "lhdm_tuning_get")
    return list(table)


def tuning_set(values):
    table = (C.c_int32 * TUNE_BUCKETS)(*values)
    _check(lib().lhdm_tuning_set(table), "lhdm_tuning_set")
