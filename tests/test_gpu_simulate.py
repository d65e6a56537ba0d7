"""Simulation through the C ABI (gp_rng_normal, gp_simulate,
gp_simulate_conditional) against the oracle.

  normals        the device's Philox4x64-10 / Box-Muller draws equal the
                 oracle's (same counters, keys and streams) to 1e-13 (the
                 two sides' log / sin / cos differ in the last bits; any
                 difference in the generator's words would not be close).
  unconditional  mu + L e_c against the oracle's realisations with its own
                 factor: 1e-11.
  conditional    posterior realisations at new locations against the
                 oracle's: 1e-8 (the posterior covariance is ill conditioned
                 when new locations are close to each other); a singular
                 posterior covariance (two equal new locations) reports
                 d_info = 2 and NaN realisations, as the oracle does.
  larger n       at n = 16,384 every realisation back-solved with the factor
                 returns its own normals (L^{-1}(Z - mu) = e) to 1e-9.
"""
import numpy as np
import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import dev, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


@pytest.mark.parametrize("n,r,stream,first", [(1001, 7, 0, 3), (4, 1, 1, 0), (9, 3, 5, 1 << 40)])
def test_normals_match_oracle(g, orc, n, r, stream, first):
    out = torch.empty(r, n, dtype=torch.float64, device="cuda")
    g.gp_rng_normal(n, r, 31337, stream, first, out, n)
    ref = orc.normals(n, r, 31337, stream=stream, first=first)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kern,n,r", [("matern32", 777, 5), ("exp", 130, 2)])
def test_simulate_matches_oracle(g, orc, kern, n, r):
    x = inputs.uniform_points(n, 70000 + n)
    s2, rho, tau2, mu = 1.4, 0.1, 0.05, -0.3
    Z = g.simulate(dev(x), kern, s2, rho, tau2, r, seed=99, first=2, mu=mu)
    L = orc.cholesky(orc.cov_fill(x, kern, s2, rho, tau2))
    ref = orc.simulate(L, r, seed=99, first=2, mu=mu)
    np.testing.assert_allclose(Z.cpu().numpy(), ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("kern,n,m,r", [("exp", 600, 150, 4), ("matern32", 257, 33, 3)])
def test_conditional_matches_oracle(g, orc, kern, n, m, r):
    x = inputs.uniform_points(n, 71000 + n)
    y = inputs.std_normal(n, 71100 + n)
    xs = inputs.uniform_points(m, 71200 + m)
    s2, rho, tau2, mu = 1.1, 0.1, 0.08, 0.2
    Z, info = g.simulate_conditional(dev(x), dev(y), dev(xs), kern, s2, rho, tau2, r, seed=5,
                                     first=1, mu=mu)
    lk = orc.loglik(x, y, kern, s2, rho, tau2, mu=mu, want_L=True)
    ref = orc.simulate_conditional(x, xs, kern, s2, rho, lk["L"], lk["alpha"], r, seed=5, first=1,
                                   mu_new=mu)
    np.testing.assert_allclose(Z.cpu().numpy(), ref, rtol=0, atol=1e-8)


def test_conditional_singular_posterior(g, orc):
    n = 200
    x = inputs.uniform_points(n, 72000)
    y = inputs.std_normal(n, 72001)
    xs = np.array([[0.5, 0.5], [0.5, 0.5], [0.1, 0.9]])
    Z, info = g.simulate_conditional(dev(x), dev(y), dev(xs), "exp", 1.0, 0.2, 0.1, 2, seed=1,
                                     check=False)
    torch.cuda.synchronize()
    assert int(info.item()) == 2
    assert torch.all(torch.isnan(Z))
    lk = orc.loglik(x, y, "exp", 1.0, 0.2, 0.1, want_L=True)
    with pytest.raises(orc.OracleNotPD) as e:
        orc.simulate_conditional(x, xs, "exp", 1.0, 0.2, lk["L"], lk["alpha"], 2, seed=1)
    assert e.value.info == 2


def test_simulate_backsolve_recovers_normals(g):
    p = inputs.config4(16384)
    n, r = p.n, 8
    x = dev(p.x)
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    lk = g.loglik(x, zero, p.kernel, p.s2, p.rho, p.tau2, precision="fp64")
    np_ = g.gp_padded_order(n)
    L = lk["ws"][: np_ * np_ * 8].view(torch.float64)
    Z = torch.empty(r, n, dtype=torch.float64, device="cuda")
    ws = torch.empty(g.gp_simulate_workspace_bytes(n, r), dtype=torch.uint8, device="cuda")
    g.gp_simulate(L, n, np_, r, 2024, 0, 0.5, Z, n, ws)
    E = torch.empty(r, n, dtype=torch.float64, device="cuda")
    g.gp_rng_normal(n, r, 2024, 0, 0, E, n)
    for c in range(r):
        v = torch.empty(n, dtype=torch.float64, device="cuda")
        g.gp_backsolve(L, n, np_, 0, (Z[c] - 0.5).contiguous(), v)
        torch.cuda.synchronize()
        err = (v - E[c]).abs().max().item()
        assert err <= 1e-9 * E[c].abs().max().item(), (c, err)
