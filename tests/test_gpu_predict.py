"""Kriging prediction (gp_predict) through the C ABI.

Against the oracle (mean and variance at every new location): the FP64
form at 1e-10 (mean relative to the largest mean, variance relative to
sigma2), the mixed form's factor at its 1e-6 bound on the variance (alpha is
refined to FP64 accuracy, so the mean is held to 1e-9).  Sizes span several
tiles with ragged tails, and more new locations than one variance chunk
(2048).

At the paper's scale (n = 67,275 training points, the clustered config-3
recipe, mixed form) no oracle can solve, so two identities that hold at any
size are checked instead.  At a training location x_i the cross covariance
is the column of C without its nugget, so
    mean_i = y_i - tau2 alpha_i    (up to the solve's residual C alpha - r)
    var_i  = tau2 - tau2^2 (C^{-1})_ii,
the first over all 67,275 training locations (the matrix-free mean at full
size), the second on a sample, with (C^{-1})_ii from gp_loglik_grad.
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


@pytest.mark.parametrize("precision,tm,tv", [("fp64", 1e-10, 1e-10), ("mixed_f16", 1e-9, 1e-6)])
@pytest.mark.parametrize("kern,n,m", [("matern32", 1500, 2500), ("exp", 777, 300),
                                      ("matern52", 1, 5)])
def test_predict_matches_oracle(g, orc, precision, tm, tv, kern, n, m):
    x = inputs.uniform_points(n, 60000 + n)
    y = inputs.std_normal(n, 60100 + n)
    xs = inputs.uniform_points(m, 60200 + m)
    s2, rho, tau2, mu = 1.3, 0.07, 0.08, 0.25
    ref = orc.predict_from_data(x, y, xs, kern, s2, rho, tau2, mu=mu, mu_new=mu)
    r = g.predict(dev(x), dev(y), dev(xs), kern, s2, rho, tau2, mu=mu, precision=precision)
    mean, var = r["mean"].cpu().numpy(), r["var"].cpu().numpy()
    assert np.max(np.abs(mean - ref["mean"])) <= tm * np.max(np.abs(ref["mean"]))
    assert np.max(np.abs(var - ref["var"])) <= tv * s2


def test_predict_mean_only_and_failure(g, orc):
    n, m = 640, 129
    x = inputs.uniform_points(n, 61000)
    y = inputs.std_normal(n, 61001)
    xs = inputs.uniform_points(m, 61002)
    ref = orc.predict_from_data(x, y, xs, "exp", 1.0, 0.1, 0.1, want_var=False)
    r = g.predict(dev(x), dev(y), dev(xs), "exp", 1.0, 0.1, 0.1, want_var=False)
    assert r["var"] is None
    assert np.max(np.abs(r["mean"].cpu().numpy() - ref["mean"])) <= 1e-10 * np.max(np.abs(ref["mean"]))
    # a non-finite new location: d_info = -2, every output NaN
    xs_bad = xs.copy()
    xs_bad[7, 1] = float("inf")
    lk = g.loglik(dev(x), dev(y), "exp", 1.0, 0.1, 0.1)
    np_ = g.gp_padded_order(n)
    mean = torch.empty(m, dtype=torch.float64, device="cuda")
    var = torch.empty(m, dtype=torch.float64, device="cuda")
    ws = torch.empty(g.gp_predict_workspace_bytes(n, m, True), dtype=torch.uint8, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_predict(dev(x), n, dev(xs_bad), m, g.params("exp", 1.0, 0.1, 0.1), lk["alpha"],
                 lk["ws"][: np_ * np_ * 8].view(torch.float64), np_, 0.0, mean, var, ws, info)
    torch.cuda.synchronize()
    assert int(info.item()) == -2
    assert torch.all(torch.isnan(mean)) and torch.all(torch.isnan(var))


def test_predict_identities_at_full_size(g):
    p = inputs.config3()
    n = p.n
    x, y = dev(p.x), dev(p.z)  # y: any data vector; the identities hold for all y
    np_ = g.gp_padded_order(n)
    ws = g.workspace(n, "mixed_f16", want_grad=True)
    lk = g.loglik(x, y, p.kernel, p.s2, p.rho, p.tau2, precision="mixed_f16", ws=ws)
    alpha = lk["alpha"]
    prm = g.params(p.kernel, p.s2, p.rho, p.tau2)
    # the mean at every training location (m = n, matrix-free)
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_predict(x, n, x, n, prm, alpha, None, np_, 0.0, mean, None, None, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    d = (mean - (y - p.tau2 * alpha)).abs().max().item()
    assert d <= 1e-9 * torch.linalg.vector_norm(y).item(), d
    # the variance at sampled training locations, against (C^{-1})_ii
    rows = np.array([0, 1, 4095, 33333, n - 1])
    xs = x[torch.as_tensor(rows, device="cuda")].contiguous()
    var = torch.empty(len(rows), dtype=torch.float64, device="cuda")
    mean_s = torch.empty(len(rows), dtype=torch.float64, device="cuda")
    pws = torch.empty(g.gp_predict_workspace_bytes(n, len(rows), True), dtype=torch.uint8,
                      device="cuda")
    g.gp_predict(x, n, xs, len(rows), prm, alpha, ws[: np_ * np_ * 8].view(torch.float64), np_,
                 0.0, mean_s, var, pws, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    var = var.cpu().numpy()
    g.loglik_grad(x, y, p.kernel, p.s2, p.rho, p.tau2, precision="mixed_f16", ws=ws)
    W = g.factor_view(ws, n)  # lower triangle of C^{-1}, column-major
    wii = W[torch.as_tensor(rows, device="cuda"), torch.as_tensor(rows, device="cuda")].cpu().numpy()
    ref = p.tau2 - p.tau2 ** 2 * wii
    assert np.max(np.abs(var - ref)) <= 1e-6 * p.tau2, (var, ref)
