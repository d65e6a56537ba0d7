"""The paper's example model (gp_loglik_product) through the C ABI: product
Matern nu = 2 in (phase, log wavelength), a random effect per phase and
known per-point variances (Sec. 4.2), against the oracle.

Inputs: the shape of the paper's data set (25 phases, an even log-wavelength
grid, measurement variances ~1e-5) at smaller sizes, with the paper's fitted
parameters (Sec. 4.3).  Tolerances: the FP64 and FP64-grade forms at the
FP64 bar (1e-10 on loglik and alpha, 1e-9 on the gradient), the mixed form
at its 1e-6 bound.  Failures: a negative or non-finite variance reports
d_info = -2.  At larger n, where the oracle is too slow, the exact identity
g_log s2 + g_log tau2 = (r^T alpha - sum v_i alpha_i^2 - n + sum v_i
(C^{-1})_ii) / 2 (the two derivatives of C add up to C - diag(v)).
"""
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


def case(n_t, n_w, orc):
    p = inputs.product_grid(n_t, n_w, seed=500 + n_w)
    v, rw = p.meta["v"], p.meta["rho_w"]
    # y = L z with the oracle's factor of this model
    L = orc.cholesky(orc.prod_cov_fill(p.x, p.s2, p.rho, rw, p.tau2, v=v))
    y = orc.lower_matvec(L, p.z)
    return p, v, rw, y


@pytest.mark.parametrize("precision,tl,tg", [("fp64", 1e-10, 1e-9), ("emu_fp64", 1e-10, 1e-9),
                                             ("mixed_f16", 1e-6, 1e-6)])
def test_product_matches_oracle(g, orc, precision, tl, tg):
    p, v, rw, y = case(5, 120, orc)
    ref = orc.prod_loglik_grad(p.x, y, p.s2, p.rho, rw, p.tau2, v=v, mu=0.01)
    r = g.loglik_product(dev(p.x), dev(y), p.s2, p.rho, rw, p.tau2, v=dev(v), mu=0.01,
                         precision=precision)
    out, grad = r["out"].cpu().numpy(), r["grad"].cpu().numpy()
    assert rel_err(out[0], ref["loglik"]) < tl, (out[0], ref["loglik"])
    assert rel_err(out[1], ref["logdet"]) < tl
    gerr = np.max(np.abs(grad - ref["grad"])) / np.max(np.abs(ref["grad"]))
    assert gerr < tg, (grad, ref["grad"])
    assert rel_norm(r["alpha"].cpu().numpy(), ref["alpha"]) < (1e-10 if tl < 1e-9 else 1e-6)


def test_product_without_variances_and_tiny(g, orc):
    # no per-point variances (v = NULL), no random effect; and n = 1
    p, _, rw, y = case(3, 50, orc)
    ref = orc.prod_loglik_grad(p.x, y, p.s2, p.rho, rw, 0.0, v=None)
    r = g.loglik_product(dev(p.x), dev(y), p.s2, p.rho, rw, 0.0, precision="fp64")
    assert rel_err(float(r["out"][0]), ref["loglik"]) < 1e-10
    gr = r["grad"].cpu().numpy()
    assert np.max(np.abs(gr - ref["grad"])) <= 1e-9 * np.max(np.abs(ref["grad"]))
    x1, y1, v1 = p.x[:1], np.array([0.3]), np.array([1e-5])
    ref1 = orc.prod_loglik_grad(x1, y1, p.s2, p.rho, rw, p.tau2, v=v1)
    r1 = g.loglik_product(dev(x1), dev(y1), p.s2, p.rho, rw, p.tau2, v=dev(v1), precision="fp64")
    assert rel_err(float(r1["out"][0]), ref1["loglik"]) < 1e-12


def test_product_bad_variance(g, orc):
    p, v, rw, y = case(2, 40, orc)
    for bad in (-1e-6, float("nan")):
        vb = v.copy()
        vb[7] = bad
        r = g.loglik_product(dev(p.x), dev(y), p.s2, p.rho, rw, p.tau2, v=dev(vb), precision="fp64",
                             check=False)
        torch.cuda.synchronize()
        assert int(r["info"].item()) == -2
        assert np.all(np.isnan(r["out"].cpu().numpy()[:3]))


@pytest.mark.parametrize("precision", ["mixed_f16", "fp64"])
def test_product_scale_identity_larger(g, precision):
    p = inputs.product_grid(25, 400 if precision == "fp64" else 1200)
    n, v, rw = p.n, p.meta["v"], p.meta["rho_w"]
    y = dev(p.z) * 0.1
    r = g.loglik_product(dev(p.x), y, p.s2, p.rho, rw, p.tau2, v=dev(v), precision=precision)
    a = r["alpha"]
    W = g.factor_view(r["ws"], n)  # lower triangle of C^{-1} (column-major)
    idx = torch.arange(n, device="cuda")
    wii = W[idx, idx]
    vd = dev(v)
    rhs = 0.5 * (torch.dot(y, a) - torch.dot(vd, a * a) - n + torch.dot(vd, wii))
    gr = r["grad"].cpu().numpy()
    tol = 1e-9 if precision == "fp64" else 1e-6
    assert abs(gr[0] + gr[3] - rhs.item()) <= tol * np.max(np.abs(gr)), (gr, rhs.item())
    assert np.all(np.isfinite(gr))
