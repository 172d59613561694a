"""The NNLS solve as a differentiable layer (torch.autograd.Function).

Forward: x = argmin ||A x - b|| s.t. x >= 0 by LHDM on the GPU (lhdm_solve
for one problem, lhdm_solve_batched for a batch).  Backward: the library's
adjoint kernel (lhdm_backward / lhdm_backward_batched) on the final passive
set P, where x_P is the least-squares solution on P (section 2.1,
subproblem (6)): with g = dL/dx and R^T R u = g_P,
    dL/db = A_P u,   dL/dA_P = r u^T - (A_P u) x_P^T,   dL/dA_Z = 0.
The map is differentiable where P is locally constant (a strictly
complementary solution); this is the gradient of that local map.

Python only marshals arguments: every arithmetic step of forward and
backward runs in the library's kernels.
"""
import torch

from . import lhdm


class _Solver:
    """Owns one library context and remembers which forward its saved
    adjoint state belongs to (a later forward on the same context replaces
    that state; backward then re-runs the forward it needs, which is
    deterministic)."""

    def __init__(self, max_m, max_n, max_batch, params):
        self.ctx = lhdm.Context(max_m, max_n, max_batch)
        self.params = params
        self.token = 0      # id of the forward whose state the context holds
        self.counter = 0

    def solve(self, A, b):
        self.counter += 1
        x, _, info = self.ctx.solve(A, b, self.params)
        if info["status"] != lhdm.LHDM_OK:
            raise RuntimeError("NNLS layer forward: " + lhdm.status_string(info["status"]))
        self.token = self.counter
        return x, self.counter

    def solve_batched(self, As, bs):
        self.counter += 1
        xs, _, infos = self.ctx.solve_batched(As, bs, self.params)
        bad = [i["status"] for i in self.ctx.info_list(infos, len(As)) if i["status"] != lhdm.LHDM_OK]
        if bad:
            raise RuntimeError("NNLS layer forward: " + lhdm.status_string(bad[0]))
        self.token = self.counter
        return xs, self.counter


class NNLSFunction(torch.autograd.Function):
    """x = NNLSFunction.apply(A, b, solver) for one problem: A (m, n) float64
    on the GPU (any strides; a column-major copy is made when needed), b (m,)."""

    @staticmethod
    def forward(ctx, A, b, solver):
        Ac = A if (A.dim() == 2 and A.stride(0) == 1 and A.stride(1) >= max(1, A.shape[0])) else lhdm.colmajor(A)
        bc = b.contiguous()
        x, tok = solver.solve(Ac, bc)
        ctx.solver, ctx.tok = solver, tok
        ctx.save_for_backward(Ac, bc)
        return x

    @staticmethod
    def backward(ctx, gx):
        Ac, bc = ctx.saved_tensors
        solver = ctx.solver
        if solver.token != ctx.tok:
            x, tok = solver.solve(Ac, bc)
            ctx.tok = tok
        want_A, want_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_A or want_b):
            return None, None, None
        db, dA = solver.ctx.backward(Ac, gx.to(torch.float64).contiguous(), want_db=want_b, want_dA=want_A)
        return dA, db, None


class NNLSBatchFunction(torch.autograd.Function):
    """xs = NNLSBatchFunction.apply(A, b, solver) for a batch of equal-size
    problems in one persistent launch: A (B, m, n) float64, b (B, m)."""

    @staticmethod
    def forward(ctx, A, b, solver):
        Ac = A.transpose(1, 2).contiguous().transpose(1, 2)  # column-major per instance
        bc = b.contiguous()
        As = [Ac[i] for i in range(Ac.shape[0])]
        bs = [bc[i] for i in range(bc.shape[0])]
        xs, tok = solver.solve_batched(As, bs)
        ctx.solver, ctx.tok = solver, tok
        ctx.save_for_backward(Ac, bc)
        return torch.stack(xs) if xs else A.new_zeros((0, A.shape[2]))

    @staticmethod
    def backward(ctx, gx):
        Ac, bc = ctx.saved_tensors
        solver = ctx.solver
        As = [Ac[i] for i in range(Ac.shape[0])]
        if solver.token != ctx.tok:
            _, tok = solver.solve_batched(As, [bc[i] for i in range(bc.shape[0])])
            ctx.tok = tok
        want_A, want_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_A or want_b) or not As:
            return None, None, None
        g = gx.to(torch.float64).contiguous()
        dbs, dAs = solver.ctx.backward_batched(As, [g[i] for i in range(g.shape[0])], want_db=want_b,
                                               want_dA=want_A)
        dA = torch.stack(dAs) if want_A else None
        db = torch.stack(dbs) if want_b else None
        return dA, db, None


class NNLSLayer(torch.nn.Module):
    """min ||A x - b|| s.t. x >= 0 as a layer: forward(A, b) takes one problem
    (A (m, n), b (m,)) or a batch (A (B, m, n), b (B, m)) and returns x with
    gradients to A and b through the library's adjoint kernel.  k_max and the
    other parameters of Algorithms 2 and 3 as in lhdm.default_params."""

    def __init__(self, max_m, max_n, max_batch=0, **params):
        super().__init__()
        self.solver = _Solver(max_m, max_n, max_batch, lhdm.default_params(**params))

    def forward(self, A, b):
        if A.dim() == 2:
            return NNLSFunction.apply(A, b, self.solver)
        if A.dim() == 3:
            return NNLSBatchFunction.apply(A, b, self.solver)
        raise ValueError("A must be (m, n) or (B, m, n)")
