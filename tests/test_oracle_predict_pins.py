"""Pins of the oracle's kriging prediction (Sec. 1: the conditional mean of the
latent process at new locations and its variance; Sec. 4.3: predictions with
standard errors).  Each pin is fixed by the mathematics, not by the oracle's
own code:

  n = 1 closed form      m = mu + s2 k / (s2 + tau2) (y - mu),
                         v = s2 - (s2 k)^2 / (s2 + tau2).
  Markov property        1-D exponential covariance, tau2 = 0 (an
                         Ornstein-Uhlenbeck process observed exactly): the
                         prediction between two training points depends on
                         those two only, with phi1, phi2 the correlations to
                         the left / right neighbour and phi = phi1 phi2:
                           m = [phi1 (1 - phi2^2) y_a + phi2 (1 - phi1^2) y_b] / (1 - phi^2)
                           v = s2 (1 - phi1^2)(1 - phi2^2) / (1 - phi^2);
                         beyond the last point m = phi y_n, v = s2 (1 - phi^2).
  interpolation          tau2 = 0 at a training location: m = y_i, v = 0.
  far away               correlation below 1e-300: m = mu_new, v = s2.
  Schur complement       v_j = det(C_aug) / det(C) with C_aug the joint
                         covariance of (Y, Z(xs_j)) (numpy slogdet, LU).
  LAPACK                 m = K^T solve(C, y - mu) (numpy's solve on the
                         oracle's C and K).
"""
import math

import numpy as np
import pytest

from paper_1305_4886_gb300 import inputs


def test_predict_n1_closed_form(orc):
    x = np.array([[0.3, 0.4]])
    xs = np.array([[0.35, 0.41], [0.9, 0.1], [0.3, 0.4]])
    y = np.array([1.7])
    for kern in ["exp", "matern32", "matern52"]:
        s2, rho, tau2, mu = 1.3, 0.2, 0.25, 0.4
        r = orc.predict_from_data(x, y, xs, kern, s2, rho, tau2, mu=mu, mu_new=mu)
        for j in range(3):
            d = math.hypot(*(xs[j] - x[0]))
            k = s2 * orc.kernel(kern, d / rho)
            m = mu + k / (s2 + tau2) * (y[0] - mu)
            v = s2 - k * k / (s2 + tau2)
            assert abs(r["mean"][j] - m) <= 1e-15 * max(1.0, abs(m))
            assert abs(r["var"][j] - v) <= 1e-15 * s2


@pytest.mark.parametrize("n", [2, 7, 300])
def test_predict_markov_property(orc, n):
    """Exponential covariance in 1-D with no nugget."""
    x = inputs.exp_fill_1d(n, 777 + n)
    t = x[:, 0]
    y = inputs.std_normal(n, 778 + n)
    s2, rho = 0.8, 0.05
    rng = np.random.default_rng(n)
    a = rng.integers(0, n - 1, size=20)
    frac = rng.random(20)
    ts = np.concatenate([t[a] + frac * (t[a + 1] - t[a]), [t[-1] + 0.013, t[-1] + 0.2]])
    xs = np.stack([ts, np.zeros_like(ts)], axis=1)
    r = orc.predict_from_data(x, y, xs, "exp", s2, rho, 0.0)
    for q in range(20):
        i = a[q]
        p1 = math.exp(-(ts[q] - t[i]) / rho)
        p2 = math.exp(-(t[i + 1] - ts[q]) / rho)
        p = p1 * p2
        m = (p1 * (1 - p2 * p2) * y[i] + p2 * (1 - p1 * p1) * y[i + 1]) / (1 - p * p)
        v = s2 * (1 - p1 * p1) * (1 - p2 * p2) / (1 - p * p)
        assert abs(r["mean"][q] - m) <= 1e-9 * (1 + abs(m)), (q, r["mean"][q], m)
        assert abs(r["var"][q] - v) <= 1e-9 * s2, (q, r["var"][q], v)
    for q in (20, 21):
        p = math.exp(-(ts[q] - t[-1]) / rho)
        assert abs(r["mean"][q] - p * y[-1]) <= 1e-9 * (1 + abs(y[-1]))
        assert abs(r["var"][q] - s2 * (1 - p * p)) <= 1e-9 * s2


@pytest.mark.parametrize("kern", ["exp", "matern32", "matern52"])
def test_predict_interpolates_without_nugget(orc, kern):
    n = 120
    x = inputs.uniform_points(n, 881)
    y = inputs.std_normal(n, 882)
    idx = [0, 17, 119]
    r = orc.predict_from_data(x, y, x[idx], kern, 1.0, 0.03, 0.0, mu=0.3, mu_new=0.3)
    np.testing.assert_allclose(r["mean"], y[idx], rtol=0, atol=1e-8)
    assert np.all(np.abs(r["var"]) <= 1e-8)


def test_predict_far_away(orc):
    x = inputs.uniform_points(50, 883)
    y = inputs.std_normal(50, 884)
    xs = np.array([[1e6, 1e6], [-5e5, 3e5]])
    r = orc.predict_from_data(x, y, xs, "matern32", 2.0, 0.1, 0.1, mu=0.5, mu_new=-0.25)
    np.testing.assert_array_equal(r["mean"], [-0.25, -0.25])
    np.testing.assert_array_equal(r["var"], [2.0, 2.0])


@pytest.mark.parametrize("kern", ["exp", "matern52"])
def test_predict_schur_complement_and_lapack(orc, kern):
    n, m = 200, 9
    x = inputs.uniform_points(n, 885)
    xs = inputs.uniform_points(m, 886)
    y = inputs.std_normal(n, 887)
    s2, rho, tau2, mu = 1.2, 0.15, 0.05, 0.1
    r = orc.predict_from_data(x, y, xs, kern, s2, rho, tau2, mu=mu, mu_new=mu)
    C = orc.cov_fill(x, kern, s2, rho, tau2)
    K = orc.cross_cov(x, xs, kern, s2, rho)
    m_ref = mu + K.T @ np.linalg.solve(C, y - mu)
    np.testing.assert_allclose(r["mean"], m_ref, rtol=1e-10, atol=1e-12)
    _, ld = np.linalg.slogdet(C)
    for j in range(m):
        aug = np.block([[C, K[:, j:j + 1]], [K[:, j:j + 1].T, np.array([[s2]])]])
        sgn, lda = np.linalg.slogdet(aug)
        assert sgn > 0
        v_ref = math.exp(lda - ld)
        assert abs(r["var"][j] - v_ref) <= 1e-9 * s2, (j, r["var"][j], v_ref)


def test_cross_cov_matches_fill_columns(orc):
    """K against the columns of the fill of the joint point set (off the
    diagonal the two use the same kernel)."""
    x = inputs.uniform_points(40, 888)
    xs = inputs.uniform_points(5, 889)
    K = orc.cross_cov(x, xs, "matern32", 1.1, 0.2)
    C = orc.cov_fill(np.concatenate([x, xs]), "matern32", 1.1, 0.2, 0.0)
    np.testing.assert_array_equal(K, C[:40, 40:])
