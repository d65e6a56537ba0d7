"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties the oracle to something it cannot get right by accident:
closed forms (n = 1, n = 2, the rho -> 0 limit), an exact rational
determinant, the Markov (AR(1)) factorisation of the 1-D exponential
covariance, Bessel-function forms of the Matern kernels, LAPACK via scipy,
invariances and the trace identity of the gradient.  A dropped term, a wrong
sign, a swapped index or a transposed operand in the oracle fails at least
one of them.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1305_4886_gb300 import inputs

LOG2PI = math.log(2.0 * math.pi)
EPS = np.finfo(np.float64).eps


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# --------------------------------------------------------------------------
# kernels: the Matern family via Bessel K (Rasmussen & Williams eq. 4.14),
# k_nu(u) = 2^{1-nu}/Gamma(nu) * a^nu K_nu(a), a = sqrt(2 nu) u.
# nu = 1/2 is the exponential.  d/da[a^nu K_nu(a)] = -a^nu K_{nu-1}(a), so
# -u k'(u) = 2^{1-nu}/Gamma(nu) * a^{nu+1} K_{nu-1}(a).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name,nu", [("exp", 0.5), ("matern32", 1.5), ("matern52", 2.5)])
def test_kernel_matches_bessel_form(orc, name, nu):
    sp = pytest.importorskip("scipy.special")
    c = 2.0 ** (1.0 - nu) / math.gamma(nu)
    for u in [1e-3, 0.05, 0.3, 1.0, 2.7, 7.5, 20.0]:
        a = math.sqrt(2.0 * nu) * u
        k_ref = c * a ** nu * sp.kv(nu, a)
        dk_ref = c * a ** (nu + 1.0) * sp.kv(nu - 1.0, a)
        assert rel(orc.kernel(name, u), k_ref) < 1e-12
        assert rel(orc.kernel_dlogrho(name, u), dk_ref) < 1e-11
    assert orc.kernel(name, 0.0) == 1.0
    assert orc.kernel_dlogrho(name, 0.0) == 0.0


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
def test_n1_closed_form(orc):
    x = np.array([[0.3, 0.7]])
    for kern in ["exp", "matern32", "matern52"]:
        s2, rho, tau2, y = 1.7, 0.2, 0.3, np.array([0.9])
        r = orc.loglik(x, y, kern, s2, rho, tau2, mu=0.25)
        c = s2 + tau2
        res = y[0] - 0.25
        expect = -0.5 * math.log(2 * math.pi * c) - res ** 2 / (2 * c)
        assert rel(r["loglik"], expect) < 1e-14
        assert rel(r["logdet"], math.log(c)) < 1e-14
        assert rel(r["alpha"][0], res / c) < 1e-14


def test_n2_closed_form(orc):
    x = np.array([[0.1, 0.2], [0.4, 0.6]])
    d = 0.5  # 3-4-5 triangle scaled by 0.1
    y = np.array([0.8, -0.3])
    for kern, kfun in [("exp", lambda u: math.exp(-u)),
                       ("matern32", lambda u: (1 + math.sqrt(3) * u) * math.exp(-math.sqrt(3) * u))]:
        s2, rho, tau2 = 1.3, 0.4, 0.2
        a = s2 + tau2
        b = s2 * kfun(d / rho)
        det = a * a - b * b
        q = (a * (y[0] ** 2 + y[1] ** 2) - 2 * b * y[0] * y[1]) / det
        expect = -0.5 * math.log(det) - 0.5 * q - LOG2PI
        r = orc.loglik(x, y, kern, s2, rho, tau2)
        assert rel(r["logdet"], math.log(det)) < 1e-14
        assert rel(r["quad"], q) < 1e-14
        assert rel(r["loglik"], expect) < 1e-14
        alpha = np.array([a * y[0] - b * y[1], -b * y[0] + a * y[1]]) / det
        assert np.allclose(r["alpha"], alpha, rtol=1e-14, atol=0)


def test_rho_to_zero_limit(orc):
    """Off-diagonal correlations underflow: C = (s2 + tau2) I exactly."""
    p = inputs.config1(64)
    s2, rho, tau2 = 1.4, 1e-7, 0.3
    y = inputs.std_normal(64, 5)
    r = orc.loglik_grad(p.x, y, "matern52", s2, rho, tau2)
    c = s2 + tau2
    n = 64
    ss = float(np.sum(y * y))
    assert rel(r["loglik"], -0.5 * n * math.log(2 * math.pi * c) - ss / (2 * c)) < 1e-13
    g0 = 0.5 * s2 * ss / c ** 2 - 0.5 * n * s2 / c
    g2 = 0.5 * tau2 * ss / c ** 2 - 0.5 * n * tau2 / c
    assert rel(r["grad"][0], g0) < 1e-12
    assert abs(r["grad"][1]) < 1e-300 + 1e-12
    assert rel(r["grad"][2], g2) < 1e-12


# --------------------------------------------------------------------------
# factorisation pins
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [5, 97, 300])
def test_reconstruction(orc, n):
    p = inputs.config1(n)
    C = orc.cov_fill(p.x, "exp", 1.0, 0.1, 0.1)
    L = orc.cholesky(C)
    assert np.all(np.triu(L, 1) == 0)
    assert np.all(np.diag(L) > 0)
    err = np.linalg.norm(L @ L.T - C) / np.linalg.norm(C)
    assert err <= 4 * n * EPS


def _exact_det(M):
    """Determinant by fraction-exact Gaussian elimination."""
    A = [[Fraction(float(v)) for v in row] for row in M]
    n = len(A)
    det = Fraction(1)
    for k in range(n):
        piv = next(i for i in range(k, n) if A[i][k] != 0)
        if piv != k:
            A[k], A[piv] = A[piv], A[k]
            det = -det
        det *= A[k][k]
        for i in range(k + 1, n):
            f = A[i][k] / A[k][k]
            for j in range(k, n):
                A[i][j] -= f * A[k][j]
    return det


def _leibniz_det(M):
    n = M.shape[0]
    tot = Fraction(0)
    for perm in itertools.permutations(range(n)):
        sgn = 1
        for i in range(n):
            for j in range(i + 1, n):
                if perm[i] > perm[j]:
                    sgn = -sgn
        prod = Fraction(1)
        for i in range(n):
            prod *= Fraction(float(M[i, perm[i]]))
        tot += sgn * prod
    return tot


@pytest.mark.parametrize("n,kern", [(3, "exp"), (6, "matern32"), (8, "matern52")])
def test_logdet_bruteforce(orc, n, kern):
    x = inputs.uniform_points(n, 100 + n)
    C = orc.cov_fill(x, kern, 1.1, 0.3, 0.05)
    ex = _exact_det(C)
    if n <= 6:
        assert _leibniz_det(C) == ex
    ld = math.log(ex.numerator) - math.log(ex.denominator)
    L = orc.cholesky(C)
    assert abs(orc.logdet(L) - ld) < 1e-12 * max(1.0, abs(ld))
    r = orc.loglik(x, np.ones(n), kern, 1.1, 0.3, 0.05)
    assert abs(r["logdet"] - ld) < 1e-12 * max(1.0, abs(ld))


# --------------------------------------------------------------------------
# AR(1) / Markov factorisation of the 1-D exponential covariance (tau2 = 0):
# y_1 ~ N(0, s2), y_i | y_{i-1} ~ N(phi_i y_{i-1}, s2 (1 - phi_i^2)),
# phi_i = exp(-(t_i - t_{i-1}) / rho).  Exact and O(n), with its own
# analytic derivatives in log s2 and log rho.
# --------------------------------------------------------------------------
def _ar1_loglik_grad(t, r, s2, rho):
    ll = -0.5 * (math.log(2 * math.pi * s2) + r[0] ** 2 / s2)
    g_s2 = -0.5 * (1.0 - r[0] ** 2 / s2)
    g_rho = 0.0
    for i in range(1, len(t)):
        dt = t[i] - t[i - 1]
        phi = math.exp(-dt / rho)
        v = s2 * (1.0 - phi * phi)
        e = r[i] - phi * r[i - 1]
        ll += -0.5 * (math.log(2 * math.pi * v) + e * e / v)
        g_s2 += -0.5 * (1.0 - e * e / v)
        dphi = (dt / rho) * phi
        dv = -2.0 * s2 * phi * dphi
        de = -r[i - 1] * dphi
        g_rho += -0.5 * (dv / v + 2.0 * e * de / v - e * e * dv / (v * v))
    return ll, g_s2, g_rho


@pytest.mark.parametrize("n", [2, 40, 400])
def test_ar1_markov_factorisation(orc, n):
    x = inputs.exp_fill_1d(n, 7 + n)
    y = inputs.std_normal(n, 11 + n)
    s2, rho = 1.6, 0.05
    r = orc.loglik_grad(x, y, "exp", s2, rho, 0.0, mu=0.1)
    ll, g0, g1 = _ar1_loglik_grad(x[:, 0], y - 0.1, s2, rho)
    assert rel(r["loglik"], ll) < 1e-10
    assert rel(r["grad"][0], g0) < 1e-9
    assert rel(r["grad"][1], g1) < 1e-9
    assert r["grad"][2] == 0.0


# --------------------------------------------------------------------------
# gradient pins
# --------------------------------------------------------------------------
def test_gradient_trace_identity(orc):
    """dC/dlog s2 + dC/dlog tau2 = C, so g0 + g2 = -n/2 + 1/2 r^T alpha."""
    p = inputs.config1(150)
    y = inputs.std_normal(150, 3)
    r = orc.loglik_grad(p.x, y, "matern32", 0.8, 0.07, 0.2)
    lhs = r["grad"][0] + r["grad"][2]
    rhs = -75.0 + 0.5 * float(np.dot(y, r["alpha"]))
    assert rel(lhs, rhs) < 1e-11


@pytest.mark.parametrize("kern", ["exp", "matern32", "matern52"])
def test_gradient_central_differences(orc, kern):
    n = 120
    x = inputs.uniform_points(n, 21)
    y = inputs.std_normal(n, 22)
    th = np.array([math.log(0.9), math.log(0.15), math.log(0.08)])

    def ll(t):
        return orc.loglik(x, y, kern, math.exp(t[0]), math.exp(t[1]), math.exp(t[2]),
                          mu=0.2)["loglik"]

    g = orc.loglik_grad(x, y, kern, *np.exp(th), mu=0.2)["grad"]
    h = 1e-5
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (ll(th + e) - ll(th - e)) / (2 * h)
        assert abs(fd - g[j]) < 1e-6 * max(1.0, abs(g[j]))


def test_inverse_is_inverse(orc):
    p = inputs.config1(200)
    C = orc.cov_fill(p.x, "exp", 1.0, 0.1, 0.1)
    W = orc.inverse_from_chol(orc.cholesky(C))
    assert np.abs(W @ C - np.eye(200)).max() < 1e-11
    assert np.array_equal(W, W.T)
    X = orc.lower_inverse(orc.cholesky(C))
    assert np.all(np.triu(X, 1) == 0)
    assert np.abs(X @ orc.cholesky(C) - np.eye(200)).max() < 1e-12


def test_solves(orc):
    p = inputs.config1(180)
    C = orc.cov_fill(p.x, "matern52", 1.0, 0.1, 0.1)
    L = orc.cholesky(C)
    b = inputs.std_normal(180, 8)
    v = orc.forward(L, b)
    assert np.abs(L @ v - b).max() < 1e-12
    a = orc.backward(L, v)
    assert np.abs(L.T @ a - v).max() < 1e-12
    assert np.abs(orc.lower_matvec(L, b) - L @ b).max() < 1e-12


# --------------------------------------------------------------------------
# invariances
# --------------------------------------------------------------------------
def test_invariances(orc):
    n = 90
    x = inputs.uniform_points(n, 31)
    y = inputs.std_normal(n, 32)
    base = orc.loglik_grad(x, y, "matern52", 1.2, 0.11, 0.07)
    perm = np.random.default_rng(33).permutation(n)
    ang = 0.7
    R = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
    variants = [
        (x[perm], y[perm]),
        (x @ R.T + np.array([3.0, -1.5]), y),
        (x[:, ::-1].copy(), y),
    ]
    for xv, yv in variants:
        r = orc.loglik_grad(xv, yv, "matern52", 1.2, 0.11, 0.07)
        assert rel(r["loglik"], base["loglik"]) < 1e-11
        assert np.max(np.abs(r["grad"] - base["grad"])) < 1e-9 * np.max(np.abs(base["grad"]))


def test_constant_mean_is_shift(orc):
    p = inputs.config2(100)
    a = orc.loglik(p.x, p.y, "matern32", 1.0, 0.05, 0.05, mu=0.5)
    b = orc.loglik(p.x, p.y - 0.5, "matern32", 1.0, 0.05, 0.05)
    assert a["loglik"] == b["loglik"]


# --------------------------------------------------------------------------
# library cross-check (LAPACK through scipy/numpy on the oracle's C)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kern", ["exp", "matern32", "matern52"])
def test_lapack_crosscheck(orc, kern):
    sl = pytest.importorskip("scipy.linalg")
    n = 600
    x = inputs.uniform_points(n, 41)
    y = inputs.std_normal(n, 42)
    C = orc.cov_fill(x, kern, 1.0, 0.08, 0.1)
    r = orc.loglik(x, y, kern, 1.0, 0.08, 0.1, want_L=True)
    Lref = np.linalg.cholesky(C)
    assert np.abs(r["L"] - Lref).max() < 1e-12
    sign, ld = np.linalg.slogdet(C)
    assert sign == 1.0 and rel(r["logdet"], ld) < 1e-12
    cf = sl.cho_factor(C, lower=True)
    alpha = sl.cho_solve(cf, y)
    assert np.linalg.norm(r["alpha"] - alpha) / np.linalg.norm(alpha) < 1e-11
    assert rel(r["quad"], float(y @ alpha)) < 1e-11


# --------------------------------------------------------------------------
# failure convention: no pivoting, first failing column reported (Sec. 5)
# --------------------------------------------------------------------------
def test_not_pd_reports_column(orc):
    x = inputs.uniform_points(10, 51)
    x[6] = x[2]  # duplicate location, no nugget: C singular
    with pytest.raises(orc.OracleNotPD) as e:
        orc.loglik(x, np.ones(10), "exp", 1.0, 0.2, 0.0)
    assert e.value.info == 7
    with pytest.raises(ValueError):
        orc.loglik(x, np.ones(10), "exp", 1.0, 0.2, -0.1)


def test_cov_rows_are_rows_of_the_fill(orc):
    x = inputs.uniform_points(150, 61)
    C = orc.cov_fill(x, "matern52", 1.3, 0.08, 0.2)
    rows = np.array([0, 7, 149, 77])
    assert np.array_equal(orc.cov_rows(x, rows, "matern52", 1.3, 0.08, 0.2), C[rows])
