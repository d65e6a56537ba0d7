"""The autograd wrapper and the L-BFGS-B likelihood fit on top of gp_loglik_grad."""
import math

import numpy as np
import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import dev, rel_err, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


@pytest.mark.parametrize("precision", ["fp64", "mixed_f16"])
def test_autograd_matches_oracle_gradient(g, orc, precision):
    from paper_1305_4886_gb300.autograd import gp_marginal_loglik
    n = 700
    x = inputs.uniform_points(n, 31000)
    y = inputs.std_normal(n, 31001)
    theta = torch.tensor([math.log(1.2), math.log(0.06), math.log(0.09)], dtype=torch.float64,
                         requires_grad=True)
    ll = gp_marginal_loglik(theta, dev(x), dev(y), "matern52", precision=precision)
    ll.backward()
    ref = orc.loglik_grad(x, y, "matern52", 1.2, 0.06, 0.09)
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert rel_err(float(ll), ref["loglik"]) < tol
    gerr = np.max(np.abs(theta.grad.numpy() - ref["grad"])) / np.max(np.abs(ref["grad"]))
    assert gerr < (1e-9 if precision == "fp64" else 1e-6)


def test_mle_fit_reaches_a_stationary_point(g, orc):
    """Data drawn from a Matern 3/2 GP with known theta; the fit must raise the
    log-likelihood from the start point and end with a small gradient."""
    pytest.importorskip("scipy")
    from paper_1305_4886_gb300 import mle
    n = 900
    x = inputs.uniform_points(n, 32000)
    true = (1.0, 0.08, 0.05)
    L = orc.cholesky(orc.cov_fill(x, "matern32", *true))
    y = orc.lower_matvec(L, inputs.std_normal(n, 32001))
    start = (math.log(0.5), math.log(0.2), math.log(0.2))
    ll0 = orc.loglik(x, y, "matern32", *np.exp(start))["loglik"]
    res = mle.fit(dev(x), dev(y), "matern32", theta0=start, precision="fp64")
    assert res["loglik"] > ll0
    assert np.max(np.abs(res["grad"])) < 1e-3 * max(1.0, abs(res["loglik"])) ** 0.5
    # the fitted log-likelihood agrees with the oracle's at the fitted theta
    ref = orc.loglik(x, y, "matern32", *res["params"])
    assert rel_err(res["loglik"], ref["loglik"]) < 1e-10
