"""Log-likelihood gradient through the C ABI (gp_loglik_grad) against the
FP64 oracle's gradient, central finite differences and the trace identity.

Tolerances: FP64 form 1e-10 relative on loglik and 1e-9 on the gradient
(infinity norm relative to the gradient's infinity norm); mixed form 1e-6
relative on both (the stated bound of the mixed form).
"""
import math

import numpy as np
import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import dev, rel_err, rel_norm, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


def grad_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("n", [1, 2, 65, 300, 700, 1100])
@pytest.mark.parametrize("kern", ["exp", "matern32", "matern52"])
def test_grad_fp64_matches_oracle(g, orc, n, kern):
    x = inputs.uniform_points(n, 11000 + n)
    y = inputs.std_normal(n, 11100 + n)
    r = g.loglik_grad(dev(x), dev(y), kern, 0.9, 0.07, 0.12, mu=0.2, precision="fp64")
    ref = orc.loglik_grad(x, y, kern, 0.9, 0.07, 0.12, mu=0.2)
    out = r["out"].cpu().numpy()
    assert rel_err(out[0], ref["loglik"]) < 1e-10
    assert grad_err(r["grad"].cpu().numpy(), ref["grad"]) < 1e-9
    assert rel_norm(r["alpha"].cpu().numpy(), ref["alpha"]) < 1e-10


@pytest.mark.parametrize("n", [300, 700, 1300])
@pytest.mark.parametrize("kern", ["exp", "matern32", "matern52"])
def test_grad_mixed_matches_oracle(g, orc, n, kern):
    x = inputs.uniform_points(n, 12000 + n)
    y = inputs.std_normal(n, 12100 + n)
    r = g.loglik_grad(dev(x), dev(y), kern, 1.1, 0.05, 0.1, precision="mixed_f16")
    ref = orc.loglik_grad(x, y, kern, 1.1, 0.05, 0.1)
    out = r["out"].cpu().numpy()
    assert rel_err(out[0], ref["loglik"]) < 1e-6
    assert grad_err(r["grad"].cpu().numpy(), ref["grad"]) < 1e-6


def test_grad_central_differences(g):
    """Central differences of the device loglik in log-parameter space
    (h = 1e-5) agree with the device gradient to the FD truncation level."""
    p = inputs.config4(400)
    y = inputs.std_normal(400, 13000)
    th = np.array([0.0, math.log(0.05), math.log(0.1)])
    xd, yd = dev(p.x), dev(y)

    def ll(t):
        return float(g.loglik(xd, yd, "matern52", *np.exp(t), precision="fp64")["out"][0])

    gd = g.loglik_grad(xd, yd, "matern52", *np.exp(th), precision="fp64")["grad"].cpu().numpy()
    h = 1e-5
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (ll(th + e) - ll(th - e)) / (2 * h)
        assert abs(fd - gd[j]) < 1e-6 * max(1.0, abs(gd[j]))


def test_grad_trace_identity_device(g):
    """g_logs2 + g_logtau2 = -n/2 + r^T alpha / 2 holds for the device result."""
    n = 500
    x = inputs.uniform_points(n, 13100)
    y = inputs.std_normal(n, 13101)
    for prec, tol in [("fp64", 1e-10), ("mixed_f16", 1e-7)]:
        r = g.loglik_grad(dev(x), dev(y), "exp", 1.3, 0.1, 0.2, precision=prec)
        gr = r["grad"].cpu().numpy()
        rhs = -n / 2 + 0.5 * float(np.dot(y, r["alpha"].cpu().numpy()))
        assert rel_err(gr[0] + gr[2], rhs) < tol


def test_grad_inverse_in_workspace(g, orc):
    """After gp_loglik_grad the matrix region holds the lower triangle of C^{-1}."""
    n = 333
    x = inputs.uniform_points(n, 13200)
    y = inputs.std_normal(n, 13201)
    r = g.loglik_grad(dev(x), dev(y), "matern32", 1.0, 0.1, 0.1, precision="fp64")
    np_ = g.gp_padded_order(n)
    W = g.factor_view(r["ws"], n).cpu().numpy().T[:n, :n]
    ref = orc.inverse_from_chol(orc.cholesky(orc.cov_fill(x, "matern32", 1.0, 0.1, 0.1)))
    low = np.tril_indices(n)
    assert np.abs(W[low] - ref[low]).max() < 1e-10 * np.abs(ref).max()
