"""Seeded synthetic NNLS instances (inputs only; no solver arithmetic).

The paper measures on a 548-matrix basis-pursuit dataset that is not
available here; these generators stand in for it with dense, seeded
instances of the shapes and value distributions used for the benchmarks:
well-conditioned underdetermined sparse recovery (Gaussian A, sparse
nonnegative x0, noiseless b) and dense overdetermined problems with noise.
N(0, v) below means variance v.  Every matrix is returned as a column-major
(Fortran-order) float64 array.  Both the CUDA path's tests/benchmark and the
CPU oracle read the same arrays.
"""
import numpy as np


def _sparse_nonneg(rng, n, s, lo=0.1):
    """s nonzeros at random positions, values uniform on (lo, 1]."""
    x = np.zeros(n)
    idx = rng.choice(n, size=s, replace=False)
    x[idx] = 1.0 - rng.uniform(0.0, 1.0 - lo, size=s)
    return x


def gaussian_recovery(m, n, s, seed, unit_columns=False):
    """A ~ N(0, 1/m) (or unit-norm Gaussian columns), x0 >= 0 with s nonzeros
    uniform on (0.1, 1], b = A x0 (noiseless)."""
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, 1.0 / np.sqrt(m), size=(m, n))
    if unit_columns:
        A /= np.linalg.norm(A, axis=0, keepdims=True)
    x0 = _sparse_nonneg(rng, n, s)
    b = A @ x0
    return np.asfortranarray(A), b, x0


def small_recovery(seed):
    """256 x 512, entries N(0, 1/256), 25 nonzeros, noiseless."""
    return gaussian_recovery(256, 512, 25, seed)


def overdetermined_uniform(seed, m=4096, n=2048, noise_var=1e-4):
    """A ~ U[0,1) (m x n), x_true with half its entries zero and the rest
    uniform on (0, 1], b = A x_true + N(0, noise_var) noise."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.0, 1.0, size=(m, n))
    x = np.zeros(n)
    nz = rng.choice(n, size=n - n // 2, replace=False)
    x[nz] = 1.0 - rng.uniform(0.0, 1.0, size=nz.size)
    b = A @ x + rng.normal(0.0, np.sqrt(noise_var), size=m)
    return np.asfortranarray(A), b, x


def sparse_recovery_sweep(seed, s, m=2048, n=8192):
    """Gaussian A with unit-norm columns, x0 >= 0 with s nonzeros, noiseless."""
    return gaussian_recovery(m, n, s, seed + 7919 * s, unit_columns=True)


def batched_sizes(batch_seed=0, count=1024, m_lo=64, m_hi=512):
    """Row counts m_i of the batched uneven workload (n_i = 2 m_i)."""
    return [int(m) for m in np.random.default_rng(batch_seed).integers(m_lo, m_hi + 1, size=count)]


def batched_instance(i, m, density=0.1, noise_var=1e-3):
    """Instance i of the batched uneven workload at m rows: n = 2m,
    A ~ N(0, 1/m), x0 with density*n nonzeros uniform on (0.1, 1],
    b = A x0 + N(0, noise_var); drawn from seed 1000 + i."""
    n = 2 * m
    rng = np.random.default_rng(1000 + i)
    A = rng.normal(0.0, 1.0 / np.sqrt(m), size=(m, n))
    x0 = _sparse_nonneg(rng, n, max(1, int(round(density * n))))
    b = A @ x0 + rng.normal(0.0, np.sqrt(noise_var), size=m)
    return np.asfortranarray(A), b, x0


def batched_uneven(batch_seed=0, count=1024, m_lo=64, m_hi=512, density=0.1, noise_var=1e-3):
    """`count` independent instances, m ~ U{m_lo..m_hi}, n = 2m, A ~ N(0, 1/m),
    x0 with density*n nonzeros uniform on (0.1, 1], b = A x0 + N(0, noise_var).
    Instance i is drawn from seed 1000 + i; its size from the batch seed."""
    sizes = batched_sizes(batch_seed, count, m_lo, m_hi)
    return [batched_instance(i, m, density, noise_var) for i, m in enumerate(sizes)]


def layer_batch(count=256, m=512, n=1024, s=40, noise_var=1e-3, seed0=0):
    """Instances for the differentiable-layer workload: A ~ N(0, 1/m),
    x0 with s nonzeros uniform on (0.1, 1], b = A x0 + N(0, noise_var),
    x_target = x0 + 1e-2 * xi with xi ~ N(0, I)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        A = rng.normal(0.0, 1.0 / np.sqrt(m), size=(m, n))
        x0 = _sparse_nonneg(rng, n, s)
        b = A @ x0 + rng.normal(0.0, np.sqrt(noise_var), size=m)
        x_target = x0 + 1e-2 * rng.normal(size=n)
        out.append((np.asfortranarray(A), b, x0, x_target))
    return out


def tiny(seed, m, n, kind="gauss"):
    """Small dense instances for brute-force checks: Gaussian A and a
    Gaussian b (so the nonnegativity constraint is active)."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, n)) if kind == "gauss" else rng.uniform(size=(m, n))
    b = rng.normal(size=m)
    return np.asfortranarray(A), b


def dependent_triple(m=12, n=8, seed=0):
    """A small instance whose first DM block contains a column that is the
    sum of two others: a_1 and a_4 orthonormal (random directions), a_6 =
    a_1 + a_4 (rounded once), the other columns small Gaussian (norm about
    0.1), b = 1.2 a_1 + a_4.  Returns A, b and the indices (i1, i2, i3) with
    a_i3 = a_i1 + a_i2."""
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, 0.1 / np.sqrt(m), size=(m, n))
    Q, _ = np.linalg.qr(rng.normal(size=(m, 2)))
    A[:, 1] = Q[:, 0]
    A[:, 4] = Q[:, 1]
    A[:, 6] = A[:, 1] + A[:, 4]
    b = 1.2 * A[:, 1] + A[:, 4]
    return np.asfortranarray(A), b, (1, 4, 6)


def with_duplicate(A, c, at):
    """A with an exact copy of column c inserted at index `at`."""
    A2 = np.insert(np.asarray(A), at, np.asarray(A)[:, c], axis=1)
    return np.asfortranarray(A2)


def _conditioned(rng, m, n, kappa):
    """m x n matrix U diag(sigma) V^T with orthonormal U (m x r), V (n x r),
    r = min(m, n), singular values log-spaced from 1 down to 1/kappa, then
    columns scaled to unit norm (which moves the condition number a little;
    the generated value is of the order of kappa)."""
    r = min(m, n)
    U, _ = np.linalg.qr(rng.normal(size=(m, r)))
    V, _ = np.linalg.qr(rng.normal(size=(n, r)))
    sigma = np.logspace(0.0, -np.log10(kappa), r)
    A = (U * sigma) @ V.T
    A /= np.linalg.norm(A, axis=0, keepdims=True)
    return A


def conditioned_overdetermined(seed, m=2048, n=1024, kappa=1e6, noise_var=1e-4):
    """Ill-conditioned dense NNLS (the paper's conditioned experiment, section
    5, with condition numbers 1e5 - 1e6): A = U diag(sigma) V^T with unit-norm
    columns, x_true with half its entries zero and the rest uniform on
    (0, 1], b = A x_true + N(0, noise_var)."""
    rng = np.random.default_rng(seed + 104729 * int(round(np.log10(kappa))))
    A = _conditioned(rng, m, n, kappa)
    x = np.zeros(n)
    nz = rng.choice(n, size=n - n // 2, replace=False)
    x[nz] = 1.0 - rng.uniform(0.0, 1.0, size=nz.size)
    b = A @ x + rng.normal(0.0, np.sqrt(noise_var), size=m)
    return np.asfortranarray(A), b, x


def conditioned_recovery(seed, m=512, n=1024, s=32, kappa=1e6):
    """Sparse nonnegative recovery with an ill-conditioned A (section 5): A as
    in conditioned_overdetermined (underdetermined), x0 >= 0 with s nonzeros
    uniform on (0.1, 1], b = A x0 (noiseless)."""
    rng = np.random.default_rng(seed + 7919 * s + 104729 * int(round(np.log10(kappa))))
    A = _conditioned(rng, m, n, kappa)
    x0 = _sparse_nonneg(rng, n, s)
    return np.asfortranarray(A), A @ x0, x0


def signed_recovery(seed, m=256, n=512, s=25, unit_columns=False):
    """Signed sparse recovery (the positivity-trick experiments of section 5):
    A ~ N(0, 1/m) (or unit-norm Gaussian columns), x0 with s nonzeros of
    random sign and magnitude uniform on (0.1, 1], b = A x0 (noiseless)."""
    rng = np.random.default_rng(seed + 31337)
    A = rng.normal(0.0, 1.0 / np.sqrt(m), size=(m, n))
    if unit_columns:
        A /= np.linalg.norm(A, axis=0, keepdims=True)
    x0 = _sparse_nonneg(rng, n, s)
    x0 *= np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    return np.asfortranarray(A), A @ x0, x0


def signed_overdetermined(seed, m=700, n=350, noise_var=1e-2):
    """Signed least squares, overdetermined: A ~ N(0, 1/m), x_true ~ N(0, 1),
    b = A x_true + N(0, noise_var)."""
    rng = np.random.default_rng(seed + 4242)
    A = rng.normal(0.0, 1.0 / np.sqrt(m), size=(m, n))
    x = rng.normal(size=n)
    b = A @ x + rng.normal(0.0, np.sqrt(noise_var), size=m)
    return np.asfortranarray(A), b, x
