"""The double-float covariance evaluation of the tensor-core forms (fill,
matrix-free residual and gradient contraction all use it) against the
oracle's FP64 fill.

Bound: a double-float value carries about 48 bits.  The coordinates are split
into FP32 pairs to 2^-48 of their magnitude, so a distance d carries an
absolute error near 2^-48 |x| and the entry an error near
sigma2 |k'(a)| scale 2^-48 |x| <= 2^-44 sigma2 for the coordinates and scales
below; exp(-a) itself carries about (1 + a) 2^-46 relative.  The test asks
|C - C*| <= 2.5e-13 sigma2 + 2e-13 (1 + a) |C*| entry by entry (2^-44 is
5.7e-14), and exact agreement in structure: the diagonal, the identity
padding, and zeros only where exp(-a) < 2^-125, i.e. where C* is below
(1 + a + a^2/3) 2^-125 sigma2 <= 1e-33 sigma2 (and a > 86.9 there).
"""
import numpy as np
import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import colmajor_to_numpy, dev, require_cuda

pytestmark = pytest.mark.gpu

SCALE = {"exp": 1.0, "matern32": 3.0 ** 0.5, "matern52": 5.0 ** 0.5}


@pytest.fixture(scope="module")
def g():
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


def points(n, seed):
    x = inputs.uniform_points(n, seed)
    x[1] = x[0] + 1e-9          # a very close pair
    x[3] = x[2]                 # two distinct points at one location
    x[5] = x[4] * 1e-6          # near the origin
    x[7] = [40.0, 40.0]         # far from everything (entries flush to zero)
    return x


@pytest.mark.parametrize("kern,rho", [("exp", 0.1), ("matern32", 0.02), ("matern52", 0.05),
                                      ("matern32", 1.3)])
@pytest.mark.parametrize("n", [777, 64])
def test_df_fill_matches_oracle(g, orc, kern, rho, n):
    s2, tau2 = 1.3, 0.2
    x = points(n, 4100 + n)
    np_ = g.gp_padded_order(n)
    buf = torch.full((np_ * np_,), np.nan, dtype=torch.float64, device="cuda")
    g.gp_cov_fill(dev(x), g.params(kern, s2, rho, tau2), buf, np_, precision="mixed_f16")
    torch.cuda.synchronize()
    C = colmajor_to_numpy(buf, np_)
    ref = orc.cov_fill(x, kern, s2, rho, tau2)
    low = np.tril_indices(n, -1)
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))[low]
    a = SCALE[kern] * d / rho
    err = np.abs(C[:n, :n][low] - ref[low])
    bound = 2.5e-13 * s2 + 2e-13 * (1.0 + a) * np.abs(ref[low])
    assert np.all(err <= bound), float(np.max(err / bound))
    zero = C[:n, :n][low] == 0.0
    assert np.all(ref[low][zero] < 1e-33 * s2) and np.all(a[zero] > 86.9)
    assert np.array_equal(np.diag(C)[:n], np.full(n, s2 + tau2))
    pad = C[n:, :]
    assert np.array_equal(np.tril(pad[:, n:]), np.eye(np_ - n)) and not np.any(pad[:, :n])
