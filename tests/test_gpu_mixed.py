"""The tensor-core (tcgen05, BF16-slice) path against FP64 references.

Bounds (stated, not fixed by the paper; the paper has no mixed precision):
  trailing update C - P P^T   |err_ij| <= 1e-6 (|P| |P|^T)_ij   (row-scaled
                              3-slice split: exact leading products, FP32
                              accumulation of the five smaller ones)
  mixed factor L              max |L - L*| <= 1e-5 max |L*|
  mixed loglik                1e-6 relative (the target bound for the mixed
                              form), alpha after refinement 1e-9 relative
"""
import numpy as np
import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import colmajor_to_numpy, dev, rel_err, rel_norm, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


@pytest.mark.parametrize("m,k", [(128, 64), (300, 100), (1000, 512), (513, 384)])
def test_tc_syrk_matches_fp64(g, m, k):
    rng = np.random.default_rng(m * 7 + k)
    P = rng.standard_normal((m, k))
    C0 = rng.standard_normal((m, m))
    C0 = C0 + C0.T
    ref = C0 - P @ P.T
    bound = np.abs(P) @ np.abs(P).T
    Cd = dev(C0.T.copy())          # column-major: storage (j, i)
    Pd = dev(P.T.copy())
    ws = torch.empty(g.gp_syrk_workspace_bytes(m, k, "mixed_f16"), dtype=torch.uint8,
                     device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_syrk_lower(Cd.view(-1), m, Pd.view(-1), m, m, k, "mixed_f16", ws, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    C = Cd.cpu().numpy().T
    low = np.tril_indices(m)
    err = np.abs(C - ref)[low] / bound[low]
    assert err.max() <= 1e-6, err.max()
    up = np.triu_indices(m, 1)
    assert np.array_equal(C[up], C0[up])  # upper triangle untouched
    # the FP64 CUDA-core variant of the same step
    Cd = dev(C0.T.copy())
    g.gp_syrk_lower(Cd.view(-1), m, Pd.view(-1), m, m, k, "fp64", None, info)
    C = Cd.cpu().numpy().T
    assert (np.abs(C - ref)[low] / bound[low]).max() <= 1e-13


@pytest.mark.parametrize("n", [100, 600, 1100, 1600])
def test_mixed_chol_matches_oracle(g, orc, n):
    x = inputs.uniform_points(n, 7000 + n)
    np_ = g.gp_padded_order(n)
    buf = torch.empty(np_ * np_, dtype=torch.float64, device="cuda")
    g.gp_cov_fill(dev(x), g.params("matern32", 1.0, 0.05, 0.1), buf, np_)
    ws = torch.empty(max(1, g.gp_chol_workspace_bytes(n, "mixed_f16")), dtype=torch.uint8,
                     device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_chol(buf, n, np_, "mixed_f16", ws, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    L = np.tril(colmajor_to_numpy(buf, np_))
    ref = orc.cholesky(orc.cov_fill(x, "matern32", 1.0, 0.05, 0.1))
    assert np.abs(L[:n, :n] - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.array_equal(L[n:, n:], np.eye(np_ - n))


@pytest.mark.parametrize("n", [100, 700, 1300])
@pytest.mark.parametrize("kern", ["exp", "matern32", "matern52"])
def test_mixed_loglik_matches_oracle(g, orc, n, kern):
    x = inputs.uniform_points(n, 8000 + n)
    y = inputs.std_normal(n, 8100 + n)
    r = g.loglik(dev(x), dev(y), kern, 1.2, 0.06, 0.08, mu=0.1, precision="mixed_f16")
    out = r["out"].cpu().numpy()
    ref = orc.loglik(x, y, kern, 1.2, 0.06, 0.08, mu=0.1)
    assert rel_err(out[0], ref["loglik"]) <= 1e-6
    assert rel_norm(r["alpha"].cpu().numpy(), ref["alpha"]) <= 1e-9
    assert out[3] <= 1e-10


def test_mixed_not_pd(g):
    n = 700
    x = inputs.uniform_points(n, 9000)
    np_ = g.gp_padded_order(n)
    buf = torch.empty(np_ * np_, dtype=torch.float64, device="cuda")
    g.gp_cov_fill(dev(x), g.params("exp", 1.0, 0.1, 0.1), buf, np_)
    k = 600  # in the second outer block
    buf[k + k * np_] = -5.0
    ws = torch.empty(g.gp_chol_workspace_bytes(n, "mixed_f16"), dtype=torch.uint8, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_chol(buf, n, np_, "mixed_f16", ws, info)
    torch.cuda.synchronize()
    assert int(info.item()) == k + 1
