"""Parity at the workloads' full sizes, where the oracle cannot factor the
whole matrix: sampled outputs the oracle computes row by row, and properties
that hold at any size.

  n = 16,384 (Matern 3/2, mu = 0.5, FP64 path): sampled entries of L L^T
      against C within the Cholesky backward-error bound
      |C - L L^T|_ij <= gamma_{n+1} sqrt(C_ii C_jj) (plus the test's own dot
      product, gamma_n); sampled residual rows of C alpha = r within
      gamma_{3n} sqrt(C_ii) sum_j sqrt(C_jj) |alpha_j| (the bound for two
      triangular solves with the computed factor); logdet = 2 sum log L_ii;
      the mixed form within 1e-6 of the FP64 log-likelihood.
  n = 67,275 (clustered Matern 3/2, the mixed form): sampled entries of
      L L^T within 1e-6 sqrt(C_ii C_jj) (FP32 rounding of each folded
      trailing update, 6e-8 of the row norms, with a 16x margin); sampled
      residual rows no larger than the refinement's stopping norm.
  n = 67,275, loglik + gradient: the mixed form against the FP64-grade
      five-slice form (itself pinned to the oracle at small n): loglik
      within 1e-8 and gradient within 1e-6 (max norm), plus the identity
      below.
  n = 32,768 (Matern 5/2, the mixed form): the exact identity
      dl/dlog s2 + dl/dlog tau2 = (q - n) / 2 (the two derivatives of C sum
      to C) within 2e-5 max|grad|, and dl/dlog rho against a central difference of the FP64
      log-likelihood (h = 1e-4, 1e-5 relative).
"""
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


def factor_rows(g, ws, n, rows):
    """Rows of L (n entries each) from the column-major factor in the workspace."""
    F = g.factor_view(ws, n)  # F[j, i] = L[i, j]
    idx = torch.as_tensor(rows, device=F.device)
    return F[:n, :][:, idx].T[:, :n].cpu().numpy()


U = 2.0 ** -53


def check_reconstruction(orc, g, p, ws, rows, tol):
    n = p.n
    Lr = factor_rows(g, ws, n, rows)
    Crow = orc.cov_rows(p.x, rows, p.kernel, p.s2, p.rho, p.tau2)
    worst = 0.0
    for a, i in enumerate(rows):
        for b, j in enumerate(rows):
            if j > i:
                continue
            lij = float(np.dot(Lr[a, : j + 1], Lr[b, : j + 1]))
            scale = math.sqrt(Crow[a, i] * Crow[b, j])
            worst = max(worst, abs(lij - Crow[a, j]) / scale)
    assert worst <= tol, worst


def residual_rows(orc, p, y, mu, alpha, rows):
    """|r_i - (C alpha)_i| at the sampled rows, with (|C| |alpha|)_i."""
    Crow = orc.cov_rows(p.x, rows, p.kernel, p.s2, p.rho, p.tau2)
    r = y[rows] - mu
    return np.abs(r - Crow @ alpha), np.abs(Crow) @ np.abs(alpha)


def test_config2_fp64_full_size(g, orc):
    p = inputs.config2()
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(p.n, 24, replace=False))
    rows[-1] = p.n - 1
    r = g.loglik(dev(p.x), dev(p.y), p.kernel, p.s2, p.rho, p.tau2, mu=p.mu, precision="fp64")
    out = r["out"].cpu().numpy()
    check_reconstruction(orc, g, p, r["ws"], rows, (2 * p.n + 1) * U)
    alpha = r["alpha"].cpu().numpy()
    res, _ = residual_rows(orc, p, p.y, p.mu, alpha, rows)
    s2t = math.sqrt(p.s2 + p.tau2)
    assert np.all(res <= 3 * p.n * U * s2t * s2t * np.sum(np.abs(alpha))), res
    F = g.factor_view(r["ws"], p.n)
    diag = torch.diagonal(F)[: p.n].cpu().numpy()
    assert rel_err(out[1], 2.0 * float(np.sum(np.log(diag)))) < 1e-12
    m = g.loglik(dev(p.x), dev(p.y), p.kernel, p.s2, p.rho, p.tau2, mu=p.mu,
                 precision="mixed_f16")
    assert rel_err(float(m["out"][0]), out[0]) < 1e-6


def test_config3_mixed_full_size(g, orc):
    p = inputs.config3()
    x, z = dev(p.x), dev(p.z)
    r = g.loglik(x, z, p.kernel, p.s2, p.rho, p.tau2, precision="mixed_f16")
    np_ = g.gp_padded_order(p.n)
    y = torch.empty_like(z)
    g.gp_mult_chol(g.factor_view(r["ws"], p.n).reshape(-1), p.n, np_, z, y)
    r = g.loglik(x, y, p.kernel, p.s2, p.rho, p.tau2, precision="mixed_f16", ws=r["ws"])
    out = r["out"].cpu().numpy()
    assert np.all(np.isfinite(out)) and out[3] <= 1e-10
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(p.n, 12, replace=False))
    check_reconstruction(orc, g, p, r["ws"], rows, 1e-6)
    yh = y.cpu().numpy()
    res, scale = residual_rows(orc, p, yh, 0.0, r["alpha"].cpu().numpy(), rows)
    # every |s_i| is below ||s|| = out[3] ||r||; 1e-14 |C||alpha| covers the
    # last-bit differences between the device's and the oracle's C
    assert np.all(res <= 1.01 * out[3] * np.linalg.norm(yh) + 1e-14 * scale), res


def test_config4_gradient_identity_and_central_difference(g):
    p = inputs.config4()
    x, z = dev(p.x), dev(p.z)
    th = np.array([0.0, math.log(0.05), math.log(0.1)])
    ws = g.workspace(p.n, "fp64")
    np_ = g.gp_padded_order(p.n)

    def ll64(t):
        return float(g.loglik(x, y, p.kernel, *np.exp(t), precision="fp64", ws=ws)["out"][0])

    g.loglik(x, z, p.kernel, *np.exp(th), precision="fp64", ws=ws)
    y = torch.empty_like(z)
    g.gp_mult_chol(g.factor_view(ws, p.n).reshape(-1), p.n, np_, z, y)
    h = 1e-4
    e = np.array([0.0, h, 0.0])
    fd = (ll64(th + e) - ll64(th - e)) / (2 * h)
    del ws
    torch.cuda.empty_cache()
    r = g.loglik_grad(x, y, p.kernel, *np.exp(th), precision="mixed_f16")
    gd = r["grad"].cpu().numpy()
    out = r["out"].cpu().numpy()
    assert abs(gd[0] + gd[2] - 0.5 * (out[2] - p.n)) <= 2e-5 * np.max(np.abs(gd))
    assert abs(fd - gd[1]) <= 1e-5 * np.max(np.abs(gd)), (fd, gd)


def test_config3_gradient_full_size(g):
    p = inputs.config3()
    x, z = dev(p.x), dev(p.z)
    ws = g.workspace(p.n, "mixed_f16", want_grad=True)
    g.loglik(x, z, p.kernel, p.s2, p.rho, p.tau2, precision="mixed_f16", ws=ws)
    y = torch.empty_like(z)
    g.gp_mult_chol(g.factor_view(ws, p.n).reshape(-1), p.n, g.gp_padded_order(p.n), z, y)
    a = g.loglik_grad(x, y, p.kernel, p.s2, p.rho, p.tau2, precision="mixed_f16", ws=ws)
    ao, ag = a["out"].cpu().numpy(), a["grad"].cpu().numpy()
    del ws, a
    torch.cuda.empty_cache()
    b = g.loglik_grad(x, y, p.kernel, p.s2, p.rho, p.tau2, precision="emu_fp64")
    bo, bg = b["out"].cpu().numpy(), b["grad"].cpu().numpy()
    assert np.all(np.isfinite(ag)) and np.all(np.isfinite(bg))
    assert rel_err(ao[0], bo[0]) < 1e-8
    assert np.max(np.abs(ag - bg)) <= 1e-6 * np.max(np.abs(bg)), (ag, bg)
    for o, gr in ((ao, ag), (bo, bg)):
        assert abs(gr[0] + gr[2] - 0.5 * (o[2] - p.n)) <= 2e-5 * np.max(np.abs(gr))
