"""Parity of the FP64 CUDA path with the oracle, through the C ABI.

Tolerances (FP64 on both sides, different summation orders):
  fill entries        1e-13 relative (one-ulp differences inside exp)
  L entries           1e-11 x max|L|
  loglik              1e-10 relative
  alpha               1e-10 relative 2-norm
Sizes span one to many 64-row tiles with ragged tails (n not a multiple of
the 128 padding).
"""
import math

import numpy as np
import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import colmajor_to_numpy, dev, rel_err, rel_norm, require_cuda

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 31, 33, 64, 127, 129, 257, 500]
KERNS = ["exp", "matern32", "matern52"]


@pytest.fixture(scope="module")
def g():
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


@pytest.mark.parametrize("n", [1, 3, 64, 129, 300])
@pytest.mark.parametrize("kern", KERNS)
def test_fill_matches_oracle(g, orc, n, kern):
    x = inputs.uniform_points(n, 1000 + n)
    np_ = g.gp_padded_order(n)
    buf = torch.full((np_ * np_,), 7.0, dtype=torch.float64, device="cuda")
    g.gp_cov_fill(dev(x), g.params(kern, 1.3, 0.07, 0.2), buf, np_)
    torch.cuda.synchronize()
    C = colmajor_to_numpy(buf, np_)
    ref = orc.cov_fill(x, kern, 1.3, 0.07, 0.2)
    low = np.tril_indices(n)
    assert np.all(np.abs(C[:n, :n][low] - ref[low]) <= 1e-13 * np.abs(ref[low]) + 1e-300)
    # padding is the identity (lower part)
    pad = np.tril(C[n:, :], 0)
    if np_ > n:
        assert np.all(pad[:, :n] == 0.0)
        assert np.array_equal(np.tril(C[n:, n:]), np.eye(np_ - n))


@pytest.mark.parametrize("n", SIZES)
def test_chol_matches_oracle(g, orc, n):
    x = inputs.uniform_points(n, 2000 + n)
    np_ = g.gp_padded_order(n)
    buf = torch.empty(np_ * np_, dtype=torch.float64, device="cuda")
    prm = g.params("matern32", 1.0, 0.1, 0.05)
    g.gp_cov_fill(dev(x), prm, buf, np_)
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_chol(buf, n, np_, "fp64", None, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    L = np.tril(colmajor_to_numpy(buf, np_))
    ref = orc.cholesky(orc.cov_fill(x, "matern32", 1.0, 0.1, 0.05))
    assert np.abs(L[:n, :n] - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.array_equal(L[n:, n:], np.eye(np_ - n))
    assert np.all(L[n:, :n] == 0.0)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kern", KERNS)
def test_loglik_matches_oracle(g, orc, n, kern):
    x = inputs.uniform_points(n, 3000 + n)
    y = inputs.std_normal(n, 3100 + n)
    mu = 0.3 if n % 2 else None
    r = g.loglik(dev(x), dev(y), kern, 1.1, 0.08, 0.07, mu=mu)
    out = r["out"].cpu().numpy()
    ref = orc.loglik(x, y, kern, 1.1, 0.08, 0.07, mu=mu)
    assert rel_err(out[0], ref["loglik"]) < 1e-10
    assert abs(out[1] - ref["logdet"]) < 1e-10 * max(1.0, abs(ref["logdet"]))
    assert rel_err(out[2], ref["quad"]) < 1e-10
    assert rel_norm(r["alpha"].cpu().numpy(), ref["alpha"]) < 1e-10


def test_config1_full_size(g, orc):
    """Exponential, n = 1024, y = L z with the oracle's factor."""
    p = inputs.config1()
    ref_L = orc.cholesky(orc.cov_fill(p.x, p.kernel, p.s2, p.rho, p.tau2))
    y = orc.lower_matvec(ref_L, p.z)
    ref = orc.loglik(p.x, y, p.kernel, p.s2, p.rho, p.tau2)
    r = g.loglik(dev(p.x), dev(y), p.kernel, p.s2, p.rho, p.tau2)
    out = r["out"].cpu().numpy()
    assert rel_err(out[0], ref["loglik"]) < 1e-10
    assert rel_err(out[1], ref["logdet"]) < 1e-10
    assert rel_norm(r["alpha"].cpu().numpy(), ref["alpha"]) < 1e-10
    np_ = g.gp_padded_order(p.n)
    L = np.tril(colmajor_to_numpy(g.factor_view(r["ws"], p.n).reshape(-1), np_))[: p.n, : p.n]
    assert np.abs(L - ref_L).max() <= 1e-11 * np.abs(ref_L).max()


@pytest.mark.parametrize("n", [1, 65, 300])
def test_backsolve_and_mult_chol(g, orc, n):
    x = inputs.uniform_points(n, 4000 + n)
    np_ = g.gp_padded_order(n)
    buf = torch.empty(np_ * np_, dtype=torch.float64, device="cuda")
    g.gp_cov_fill(dev(x), g.params("exp", 1.0, 0.2, 0.1), buf, np_)
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_chol(buf, n, np_, "fp64", None, info)
    b = inputs.std_normal(n, 4100 + n)
    ref_L = orc.cholesky(orc.cov_fill(x, "exp", 1.0, 0.2, 0.1))
    bd = dev(b)
    out = torch.empty_like(bd)
    g.gp_backsolve(buf, n, np_, 0, bd, out)
    assert rel_norm(out.cpu().numpy(), orc.forward(ref_L, b)) < 1e-11
    g.gp_backsolve(buf, n, np_, 1, bd, out)
    assert rel_norm(out.cpu().numpy(), orc.backward(ref_L, b)) < 1e-11
    inplace = bd.clone()
    g.gp_backsolve(buf, n, np_, 0, inplace, inplace)
    assert rel_norm(inplace.cpu().numpy(), orc.forward(ref_L, b)) < 1e-11
    g.gp_mult_chol(buf, n, np_, bd, out)
    assert rel_norm(out.cpu().numpy(), orc.lower_matvec(ref_L, b)) < 1e-13


def test_not_positive_definite_reports_column(g):
    """No pivoting (Sec. 5): a negative pivot at column k gives info = k + 1."""
    n = 200
    x = inputs.uniform_points(n, 5000)
    np_ = g.gp_padded_order(n)
    buf = torch.empty(np_ * np_, dtype=torch.float64, device="cuda")
    g.gp_cov_fill(dev(x), g.params("exp", 1.0, 0.1, 0.1), buf, np_)
    k = 137
    buf[k + k * np_] = -1.0
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_chol(buf, n, np_, "fp64", None, info)
    torch.cuda.synchronize()
    assert int(info.item()) == k + 1


def test_nonfinite_inputs_flagged(g):
    n = 100
    x = inputs.uniform_points(n, 6000)
    y = inputs.std_normal(n, 6001)
    xb = x.copy()
    xb[17, 1] = float("nan")
    r = g.loglik(dev(xb), dev(y), "exp", 1.0, 0.1, 0.1, check=False)
    assert int(r["info"].item()) == -2
    assert math.isnan(float(r["out"][0]))
    yb = y.copy()
    yb[3] = float("inf")
    r = g.loglik(dev(x), dev(yb), "exp", 1.0, 0.1, 0.1, check=False)
    assert int(r["info"].item()) == -2
    with pytest.raises(g.GpDeviceError):
        g.loglik(dev(x), dev(yb), "exp", 1.0, 0.1, 0.1)


def test_fill_exponent_range(g, orc):
    """Kernel arguments a spread over [0, 1600] (the device exp's whole range,
    including the flush to zero near the FP64 underflow).

    exp(-a) has condition number a, so one ulp of a (the oracle divides by
    rho, the device multiplies by 1/rho) moves it by a*eps relative: against
    the oracle the bound is 1e-13 + 8 a eps.  Against numpy's exp at the very
    same a (formed like the device: sqrt of the squared differences times
    c/rho), the device exp itself must hold 1e-13 relative.  Entries below
    1e-290 must be below 1e-290 on the device too."""
    n = 700
    t = np.linspace(0.0, 1.0, n)
    x = np.stack([t * t, np.zeros(n)], axis=1)  # uneven spacing: many distinct a
    rho = 1.0 / 720.0
    np_ = g.gp_padded_order(n)
    buf = torch.empty(np_ * np_, dtype=torch.float64, device="cuda")
    low = np.tril_indices(n, -1)
    d = np.sqrt((x[:, None, 0] - x[None, :, 0]) ** 2 + (x[:, None, 1] - x[None, :, 1]) ** 2)[low]
    eps = np.finfo(np.float64).eps
    for kern, c in [("exp", 1.0), ("matern32", math.sqrt(3.0)), ("matern52", math.sqrt(5.0))]:
        g.gp_cov_fill(dev(x), g.params(kern, 1.0, rho, 0.0), buf, np_)
        torch.cuda.synchronize()
        C = colmajor_to_numpy(buf, np_)[:n, :n][low]
        a = d * (c / rho)
        e = np.exp(-a)
        same_a = {"exp": e, "matern32": (a * e + e),
                  "matern52": (1.0 + a + a * a * (1.0 / 3.0)) * e}[kern]
        ref = orc.cov_fill(x, kern, 1.0, rho, 0.0)[low]
        big = np.abs(ref) > 1e-290
        assert np.all(np.abs(C[big] - same_a[big]) <= 1e-13 * np.abs(same_a[big]))
        assert np.all(np.abs(C[big] - ref[big]) <= (1e-13 + 8 * eps * a[big]) * np.abs(ref[big]))
        assert np.all(np.abs(C[~big]) <= 1e-290)
