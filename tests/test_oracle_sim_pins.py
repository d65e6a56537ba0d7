"""Pins of the oracle's simulation (Sec. 1: unconditional and conditional
realisations; Sec. 2.3.2: the Cholesky factor times standard normals;
Sec. 4.3: posterior realisations).

  generator     Philox4x64-10 words equal numpy's Philox bit generator (the
                same published generator; numpy's raw output for counter c
                is the block function at c + 1), for many counters and keys.
  normals       the Box-Muller draws are standard normal: mean, variance,
                fourth moment and a Kolmogorov-Smirnov test on 2^20 draws;
                distinct realisations and streams are uncorrelated.
  simulate      realisation c equals mu + L e_c (numpy's matmul on the
                oracle's own draws), and the sample covariance of 40,000
                realisations matches C within its sampling error.
  conditional   1-D exponential covariance without nugget (Ornstein-
                Uhlenbeck), one new location between two training points:
                the posterior is N(m, v) with the closed-form m, v of the
                Markov property, so each realisation is m + sqrt(v) z_c with
                z_c the stream-1 normal; far from all training points the
                realisations are unconditional draws of the new locations'
                covariance.
"""
import math

import numpy as np
import pytest

from paper_1305_4886_gb300 import inputs


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(5)
    for _ in range(50):
        ctr = [int(v) for v in rng.integers(0, 2 ** 63, size=4, dtype=np.int64)]
        key = [int(v) for v in rng.integers(0, 2 ** 63, size=2, dtype=np.int64)]
        bg = np.random.Philox(counter=ctr, key=key)
        want = bg.random_raw(4)
        ctr1 = list(ctr)
        ctr1[0] += 1
        got = orc.philox4x64(ctr1, key)
        np.testing.assert_array_equal(got, want)
    # the counter carries into the next word
    bg = np.random.Philox(counter=np.array([2 ** 64 - 1, 7, 0, 0], dtype=np.uint64), key=[3, 4])
    np.testing.assert_array_equal(orc.philox4x64([0, 8, 0, 0], [3, 4]), bg.random_raw(4))


def test_normals_are_standard_normal(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    z = orc.normals(1 << 14, 64, seed=2024).ravel()
    N = z.size
    assert abs(z.mean()) < 5 / math.sqrt(N)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / N)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * math.sqrt(96.0 / N)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    a = orc.normals(4096, 2, seed=7, stream=0)
    b = orc.normals(4096, 1, seed=7, stream=1)
    for u, v in [(a[0], a[1]), (a[0], b[0])]:
        assert abs(np.corrcoef(u, v)[0, 1]) < 5 / math.sqrt(4096)
    # realisation offsets: draws of realisation first + c
    np.testing.assert_array_equal(orc.normals(33, 3, 9, first=5)[1], orc.normals(33, 1, 9, first=6)[0])


def test_simulate_is_factor_times_normals(orc):
    n = 37
    x = inputs.uniform_points(n, 990)
    L = orc.cholesky(orc.cov_fill(x, "matern32", 1.5, 0.2, 0.05))
    Z = orc.simulate(L, 6, seed=11, first=3, mu=0.7)
    E = orc.normals(n, 6, 11, first=3)
    np.testing.assert_allclose(Z, 0.7 + E @ L.T, rtol=0, atol=1e-13)


def test_simulate_covariance(orc):
    n, r = 5, 40000
    x = inputs.uniform_points(n, 991)
    C = orc.cov_fill(x, "exp", 1.2, 0.3, 0.1)
    Z = orc.simulate(orc.cholesky(C), r, seed=12)
    S = Z.T @ Z / r
    sd = np.sqrt((C ** 2 + np.outer(np.diag(C), np.diag(C))) / r)  # Wishart entry sd
    assert np.all(np.abs(S - C) < 5 * sd)


def test_conditional_markov_closed_form(orc):
    n = 40
    x = inputs.exp_fill_1d(n, 992)
    t = x[:, 0]
    y = inputs.std_normal(n, 993)
    s2, rho = 0.9, 0.04
    tn = 0.3 * t[10] + 0.7 * t[11]
    xs = np.array([[tn, 0.0]])
    lk = orc.loglik(x, y, "exp", s2, rho, 0.0, want_L=True)
    R = orc.simulate_conditional(x, xs, "exp", s2, rho, lk["L"], lk["alpha"], 8, seed=77)
    p1, p2 = math.exp(-(tn - t[10]) / rho), math.exp(-(t[11] - tn) / rho)
    p = p1 * p2
    m = (p1 * (1 - p2 * p2) * y[10] + p2 * (1 - p1 * p1) * y[11]) / (1 - p * p)
    v = s2 * (1 - p1 * p1) * (1 - p2 * p2) / (1 - p * p)
    z = orc.normals(1, 8, 77, stream=1)[:, 0]
    np.testing.assert_allclose(R[:, 0], m + math.sqrt(v) * z, rtol=0, atol=1e-9)


def test_conditional_far_away_is_unconditional(orc):
    n, m = 30, 6
    x = inputs.uniform_points(n, 994)
    y = inputs.std_normal(n, 995)
    xs = 1e4 + inputs.uniform_points(m, 996)
    lk = orc.loglik(x, y, "matern52", 1.1, 0.2, 0.1, want_L=True)
    R = orc.simulate_conditional(x, xs, "matern52", 1.1, 0.2, lk["L"], lk["alpha"], 5, seed=5,
                                 mu_new=0.4)
    Ls = orc.cholesky(orc.cov_fill(xs, "matern52", 1.1, 0.2, 0.0))
    E = orc.normals(m, 5, 5, stream=1)
    np.testing.assert_allclose(R, 0.4 + E @ Ls.T, rtol=0, atol=1e-12)


def test_conditional_not_pd_reports_column(orc):
    """Two identical new locations: the posterior covariance is singular and
    the unpivoted factorisation stops (Sec. 5)."""
    x = inputs.uniform_points(20, 997)
    y = inputs.std_normal(20, 998)
    xs = np.array([[0.5, 0.5], [0.5, 0.5]])
    lk = orc.loglik(x, y, "exp", 1.0, 0.2, 0.1, want_L=True)
    with pytest.raises(orc.OracleNotPD) as e:
        orc.simulate_conditional(x, xs, "exp", 1.0, 0.2, lk["L"], lk["alpha"], 2, seed=1)
    assert e.value.info == 2
