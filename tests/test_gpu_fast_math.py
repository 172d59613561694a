"""The solver's reciprocal (Newton-Raphson from a single-precision seed) and
square root (Goldschmidt step plus a Newton correction with the exact
remainder) against the library's correctly rounded division and square root
on the GPU: within one ulp over the normal range (both signs, mantissas and
exponents spread out, powers of two, neighbours of powers of two), and the
library's own answer at zero, subnormals, the extreme exponents, infinities
and NaN, where the routines hand over to it."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05345_gb300 import build, lhdm
    build.build()
    return lhdm


def ulps(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_normal_range_within_one_ulp(L):
    rng = np.random.default_rng(11)
    mant = rng.uniform(1.0, 2.0, 200000)
    expo = rng.integers(-990, 990, mant.size)
    x = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], mant.size)
    p2 = np.ldexp(1.0, np.arange(-990, 990))
    x = np.concatenate([x, p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), -p2])
    out = L.fast_math(torch.from_numpy(x).cuda()).cpu().numpy()
    assert ulps(out[:, 0], out[:, 1]).max() <= 1.0
    assert ulps(out[:, 2], out[:, 3]).max() <= 1.0
    # most results are the correctly rounded ones
    assert (out[:, 0] == out[:, 1]).mean() > 0.99
    assert (out[:, 2] == out[:, 3]).mean() > 0.99


def test_edge_arguments_take_the_library_route(L):
    x = np.array([0.0, -0.0, 5e-324, 1e-310, 2.0 ** -1010, 2.0 ** 1010, 1.7e308,
                  np.inf, -np.inf, np.nan])
    out = L.fast_math(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(out[:, 0], out[:, 1])
    np.testing.assert_array_equal(out[:, 2], out[:, 3])
