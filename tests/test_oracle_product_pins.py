"""Pins of the oracle's product model, the paper's example covariance
(Sec. 4.2): flux at (phase t, log wavelength w) = GP value + random effect of
the phase + measurement error of known variance,
    C_ij = s2 k(|t_i - t_j| / rho_t) k(|w_i - w_j| / rho_w)
           + tau2 [t_i == t_j] + v_i [i == j],
k the Matern correlation of smoothness 2 (Rasmussen & Williams scaling:
k(u) = a^2 K_2(a) / 2, a = 2u).

  Bessel K      the oracle's quadrature of the integral representation
                against scipy's kv, orders 1 and 2, x in [1e-10, 600].
  kernel        k and -u k'(u) against their definitions through scipy's kv
                (and k' by central differences); k(0) = 1, k = 1 - u^2 + ...
  Kronecker     on a full (phase x wavelength) grid with tau2 = 0 and a
                constant v: C = s2 K_t (x) K_w + v I, so logdet and q follow
                from the eigenvalues of the two small factors (numpy eigh).
  one phase     all points at one phase, v = 0: C = s2 K_w + tau2 1 1^T, so
                det C = det(s2 K_w)(1 + tau2 1^T (s2 K_w)^{-1} 1) and q by the
                Sherman-Morrison formula.
  n = 2         closed-form loglik for two points at one phase and at two
                phases.
  gradient      central differences in the four log parameters; the
                identity g_s2 + g_tau2 = 1/2 r^T alpha - 1/2 sum v_i alpha_i^2
                - n/2 + 1/2 sum v_i (C^{-1})_ii.
"""
import math

import numpy as np
import pytest

sp = pytest.importorskip("scipy.special")

LOG2PI = math.log(2 * math.pi)


def k_ref(u):
    u = np.asarray(u, dtype=float)
    a = 2.0 * u
    with np.errstate(invalid="ignore", divide="ignore"):
        v = 0.5 * a * a * sp.kv(2, a)
    return np.where(u == 0.0, 1.0, v)


def grid(nt, nw, seed):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(-15, 24, size=nt))
    w = np.sort(rng.uniform(8.69, 8.75, size=nw))
    return np.array([[ti, wi] for ti in t for wi in w]), t, w


def test_bessel_k_matches_scipy(orc):
    worst = 0.0
    for x in np.logspace(-10, math.log10(600), 300):  # scipy kv underflows near 700
        for nu in (1, 2):
            worst = max(worst, abs(orc.bessel_k(nu, x) - sp.kv(nu, x)) / sp.kv(nu, x))
    assert worst < 1e-13, worst


def test_matern2_kernel_and_derivative(orc):
    assert orc.matern2(0.0) == 1.0 and orc.matern2_dlogrho(0.0) == 0.0
    for u in [1e-7, 1e-4, 0.01, 0.3, 1.0, 2.5, 7.0, 20.0]:
        assert abs(orc.matern2(u) - float(k_ref(u))) <= 1e-14 * max(1e-300, float(k_ref(u))) + 1e-300
    for u in [0.01, 0.3, 1.0, 2.5, 7.0, 20.0]:
        h = 1e-5 * u
        dk = (float(k_ref(u + h)) - float(k_ref(u - h))) / (2 * h)
        assert abs(orc.matern2_dlogrho(u) - (-u * dk)) <= 1e-7 * abs(u * dk)
    # near 0: k = 1 - u^2 + O(u^4 log u), so -u k'(u) = 2 u^2 + ...
    for u in [1e-6, 1e-5]:
        assert abs(orc.matern2(u) - (1 - u * u)) < 1e-9 * u * u + 4e-16
        assert abs(orc.matern2_dlogrho(u) - 2 * u * u) < 1e-7 * u * u


def test_kronecker_structure(orc):
    nt, nw = 5, 9
    x, t, w = grid(nt, nw, 1)
    s2, rt, rw, v = 1.3, 6.0, 0.01, 0.05
    y = np.random.default_rng(2).standard_normal(nt * nw)
    Kt = k_ref(np.abs(t[:, None] - t[None, :]) / rt)
    Kw = k_ref(np.abs(w[:, None] - w[None, :]) / rw)
    lt, Ut = np.linalg.eigh(Kt)
    lw, Uw = np.linalg.eigh(Kw)
    lam = s2 * np.outer(lt, lw).ravel() + v
    yt = np.kron(Ut, Uw).T @ y
    logdet, q = np.sum(np.log(lam)), np.sum(yt * yt / lam)
    r = orc.prod_loglik_grad(x, y, s2, rt, rw, 0.0, v=np.full(nt * nw, v), want_grad=False)
    assert abs(r["logdet"] - logdet) <= 1e-10 * abs(logdet)
    assert abs(r["quad"] - q) <= 1e-10 * q
    assert abs(r["loglik"] - (-0.5 * logdet - 0.5 * q - 0.5 * nt * nw * LOG2PI)) <= 1e-10 * abs(r["loglik"])


def test_one_phase_rank_one_effect(orc):
    nw = 30
    w = np.sort(np.random.default_rng(3).uniform(0, 1, size=nw))
    x = np.stack([np.full(nw, 2.0), w], axis=1)
    s2, rw, tau2 = 0.8, 0.07, 0.3
    y = np.random.default_rng(4).standard_normal(nw)
    A = s2 * k_ref(np.abs(w[:, None] - w[None, :]) / rw)
    one = np.ones(nw)
    Ai1, Aiy = np.linalg.solve(A, one), np.linalg.solve(A, y)
    denom = 1 + tau2 * one @ Ai1
    logdet = np.linalg.slogdet(A)[1] + math.log(denom)
    q = y @ Aiy - tau2 * (one @ Aiy) ** 2 / denom
    r = orc.prod_loglik_grad(x, y, s2, 3.0, rw, tau2, want_grad=False)
    assert abs(r["logdet"] - logdet) <= 1e-9 * abs(logdet)
    assert abs(r["quad"] - q) <= 1e-9 * abs(q)


@pytest.mark.parametrize("same_phase", [True, False])
def test_two_points_closed_form(orc, same_phase):
    x = np.array([[1.0, 0.3], [1.0 if same_phase else 2.5, 0.31]])
    y = np.array([0.7, -0.4])
    v = np.array([0.02, 0.07])
    s2, rt, rw, tau2 = 1.1, 2.0, 0.05, 0.2
    kt = 1.0 if same_phase else float(k_ref(1.5 / rt))
    c12 = s2 * kt * float(k_ref(0.01 / rw)) + (tau2 if same_phase else 0.0)
    c11, c22 = s2 + tau2 + v[0], s2 + tau2 + v[1]
    det = c11 * c22 - c12 * c12
    q = (c22 * y[0] ** 2 - 2 * c12 * y[0] * y[1] + c11 * y[1] ** 2) / det
    ll = -0.5 * math.log(det) - 0.5 * q - LOG2PI
    r = orc.prod_loglik_grad(x, y, s2, rt, rw, tau2, v=v, want_grad=False)
    assert abs(r["loglik"] - ll) <= 1e-13 * abs(ll)


def test_gradient_finite_differences_and_identity(orc):
    x, _, _ = grid(4, 15, 5)
    n = x.shape[0]
    rng = np.random.default_rng(6)
    y = rng.standard_normal(n)
    v = rng.uniform(0.01, 0.05, size=n)
    th = np.log([0.9, 5.0, 0.012, 0.15])

    def ll(t):
        e = np.exp(t)
        return orc.prod_loglik_grad(x, y, e[0], e[1], e[2], e[3], v=v, want_grad=False)["loglik"]

    e = np.exp(th)
    r = orc.prod_loglik_grad(x, y, e[0], e[1], e[2], e[3], v=v)
    for j in range(4):
        d = np.zeros(4)
        d[j] = 1e-5
        fd = (ll(th + d) - ll(th - d)) / 2e-5
        assert abs(r["grad"][j] - fd) <= 1e-6 * max(1.0, np.max(np.abs(r["grad"]))), (j, r["grad"][j], fd)
    C = orc.prod_cov_fill(x, e[0], e[1], e[2], e[3], v=v)
    W = np.linalg.inv(C)
    a = r["alpha"]
    rhs = 0.5 * y @ a - 0.5 * np.sum(v * a * a) - 0.5 * n + 0.5 * np.sum(v * np.diag(W))
    assert abs(r["grad"][0] + r["grad"][3] - rhs) <= 1e-9 * max(1.0, abs(rhs))
