"""The float64 quotient of the eigen step against CUDA's division.

The noise estimate divides in float64 twice (Section 2.3): the Rayleigh
quotients v^T Sigma v / v^T v (denominators near 1) and the tail mean
tail / (D - m) (denominators 1..57).  It uses a float32 reciprocal refined by
Newton steps instead of the library division; here it must agree with CUDA's
correctly rounded a / b within two ulps over those operand ranges and a wider
sweep of magnitudes.
"""
import numpy as np
import pytest
import torch

from paper_2401_09721_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_2401_09721_gb300 import fgbd
    return fgbd


def _ulps(x, y):
    xi = x.view(np.int64)
    yi = y.view(np.int64)
    return np.abs(xi - yi)


def test_div_newton_within_two_ulps(F):
    rng = np.random.default_rng(3)
    n = 1 << 20
    a = np.concatenate([
        rng.uniform(0.0, 1e6, n // 4),                      # tail sums of eigenvalues (0..255^2 x 57)
        rng.uniform(0.0, 7e4, n // 4) * rng.uniform(0.5, 2.0, n // 4),  # Rayleigh numerators
        10.0 ** rng.uniform(-30, 30, n // 4),                # a wide sweep of magnitudes
        rng.integers(0, 1 << 40, n // 4).astype(np.float64),  # exact integers
    ])
    b = np.concatenate([
        rng.integers(1, 58, n // 4).astype(np.float64),      # D - m
        rng.uniform(0.5, 2.0, n // 4),                       # v^T v of near-unit vectors
        10.0 ** rng.uniform(-30, 30, n // 4),
        rng.integers(1, 1 << 20, n // 4).astype(np.float64),
    ])
    qn, qd = F.fgbd_debug_div(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    qn, qd = qn.cpu().numpy(), qd.cpu().numpy()
    assert np.array_equal(qd, a / b)          # CUDA's division is the correctly rounded quotient
    assert _ulps(qn, qd).max() <= 2
    # representable quotients (integers over divisors that divide them) come within one ulp
    k = rng.integers(1, 58, 4096).astype(np.float64)
    m = rng.integers(1, 1 << 30, 4096).astype(np.float64)
    qn, _ = F.fgbd_debug_div(torch.from_numpy(m * k).cuda(), torch.from_numpy(k).cuda())
    assert _ulps(qn.cpu().numpy(), m).max() <= 1
