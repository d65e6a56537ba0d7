"""The FP64-grade emulation mode (GP_EMU_FP64): five integer-valued BF16
slices, 15 slice products, exactly accumulated leading groups, double-float
pending updates.  Checked against FP64 references at FP64-class tolerances:
  trailing update   |err_ij| <= 3e-11 (|P| |P|^T)_ij   (2^-40 of the row maxima,
                    which can be ~10x the typical entry)
  loglik            1e-10 relative (the FP64 bound)
  gradient          1e-9 relative (infinity norm; the FP64 bound)
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


@pytest.mark.parametrize("m,k", [(300, 100), (1000, 512)])
def test_emu_syrk(g, m, k):
    rng = np.random.default_rng(m + 3 * k)
    P = rng.standard_normal((m, k)) * np.exp(rng.uniform(-3, 3, size=(m, 1)))
    C0 = rng.standard_normal((m, m))
    C0 = C0 + C0.T
    ref = C0 - P @ P.T
    bound = np.abs(P) @ np.abs(P).T
    Cd = dev(C0.T.copy())
    Pd = dev(P.T.copy())
    ws = torch.empty(g.gp_syrk_workspace_bytes(m, k, "emu_fp64"), dtype=torch.uint8, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gp_syrk_lower(Cd.view(-1), m, Pd.view(-1), m, m, k, "emu_fp64", ws, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    C = Cd.cpu().numpy().T
    low = np.tril_indices(m)
    err = np.abs(C - ref)[low] / bound[low]
    assert err.max() <= 3e-11, err.max()


@pytest.mark.parametrize("n", [300, 900, 1300])
@pytest.mark.parametrize("kern", ["exp", "matern32", "matern52"])
def test_emu_loglik_grad_matches_oracle(g, orc, n, kern):
    x = inputs.uniform_points(n, 50000 + n)
    y = inputs.std_normal(n, 50100 + n)
    r = g.loglik_grad(dev(x), dev(y), kern, 1.1, 0.05, 0.1, mu=0.2, precision="emu_fp64")
    ref = orc.loglik_grad(x, y, kern, 1.1, 0.05, 0.1, mu=0.2)
    out = r["out"].cpu().numpy()
    assert rel_err(out[0], ref["loglik"]) < 1e-10
    gerr = np.max(np.abs(r["grad"].cpu().numpy() - ref["grad"])) / np.max(np.abs(ref["grad"]))
    assert gerr < 1e-9, gerr
    assert rel_norm(r["alpha"].cpu().numpy(), ref["alpha"]) < 1e-10


def test_emu_clustered_matches_fp64_path(g):
    """The clustered, small-range workload (the hard case for the 3-slice form's
    gradient) against the FP64 CUDA path at n = 3000."""
    p = inputs.config3(3000)
    x, z = dev(p.x), dev(p.z)
    a = g.loglik_grad(x, z, p.kernel, p.s2, p.rho, p.tau2, precision="fp64")
    b = g.loglik_grad(x, z, p.kernel, p.s2, p.rho, p.tau2, precision="emu_fp64")
    assert rel_err(float(b["out"][0]), float(a["out"][0])) < 1e-10
    ga, gb = a["grad"].cpu().numpy(), b["grad"].cpu().numpy()
    assert np.max(np.abs(ga - gb)) / np.max(np.abs(ga)) < 1e-9
