"""Dense closed-form adjoint of the NNLS solution map (test infrastructure).

On a fixed passive set P with A_P of full column rank, the NNLS solution is
the least-squares solution on P (section 2.1, subproblem (6) with the normal
equations): x_P = (A_P^T A_P)^{-1} A_P^T b, x_Z = 0.  Differentiating that
definition for a loss L with gradient g = dL/dx gives, with
u = (A_P^T A_P)^{-1} g_P and r = b - A_P x_P,
    dL/db     = A_P u,
    dL/dA_P   = r u^T - (A_P u) x_P^T,
    dL/dA_Z   = 0.
This module writes that out with the normal-equation matrix formed
explicitly and numpy.linalg.solve as the only library step.
"""
import numpy as np


def nnls_adjoint(A, b, x, passive, g):
    A = np.asarray(A, dtype=np.float64)
    P = np.asarray(sorted(int(i) for i in passive), dtype=np.int64)
    m, n = A.shape
    dLdA = np.zeros((m, n))
    if P.size == 0:
        return np.zeros(m), dLdA
    AP = A[:, P]
    M = AP.T @ AP
    u = np.linalg.solve(M, np.asarray(g, dtype=np.float64)[P])
    r = np.asarray(b, dtype=np.float64) - AP @ np.asarray(x, dtype=np.float64)[P]
    APu = AP @ u
    dLdA[:, P] = np.outer(r, u) - np.outer(APu, np.asarray(x, dtype=np.float64)[P])
    return APu, dLdA
