"""gp_loglik_noalloc: the log-likelihood entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they need a
log-likelihood (for example code running while a stream is being captured,
or a host application that owns every device allocation).  It keeps its
scratch in a static device array, so it only serves n <= GP_NOALLOC_MAX_N.

Checked here through the C ABI:
  - two calls in a row, the largest size first and then a smaller one (so
    that the shared scratch still holds the previous call's factor at
    another leading dimension), each against gp_loglik (the workspace entry
    point, FP64) and against the oracle, within the FP64 parity tolerance of
    the other tests (1e-10 relative on loglik, logdet, q and alpha);
  - a size above the limit is rejected with GP_ERR_TOO_LARGE before any
    device work.
The test does not depend on what ran before it: it passes alone in a fresh
process and after the rest of the suite.  Its file name only makes pytest
collect it last, so that a run stopping at its first failure has already
run every other test.
"""
import ctypes

import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import dev, rel_err, rel_norm, require_cuda

pytestmark = pytest.mark.gpu

GP_ERR_TOO_LARGE = 6
NOALLOC_MAX_N = 512
S2, RHO, TAU2 = 1.1, 0.08, 0.1


def _noalloc(L, gp, x, y, prm, n, mu=None):
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    alpha = torch.empty(n, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = L.gp_loglik_noalloc(gp._f64(x), gp._f64(y), gp._f64(mu), n, ctypes.byref(prm),
                             gp._f64(out), gp._f64(alpha), gp._ptr(info), gp._stream())
    assert st == 0, st
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    return out.cpu().numpy(), alpha.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_and_oracle_twice(orc):
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    L = gp.lib()
    # the largest size first, then a smaller one over the same scratch
    cases = [(NOALLOC_MAX_N, "exp", None), (300, "matern32", 0.4)]
    for n, kern, mu in cases:
        x = inputs.uniform_points(n, 21000 + n)
        y = inputs.std_normal(n, 21100 + n)
        prm = gp.params(kern, S2, RHO, TAU2)
        xd, yd = dev(x), dev(y)
        mud = torch.full((n,), mu, dtype=torch.float64, device="cuda") if mu is not None else None
        out_na, alpha_na = _noalloc(L, gp, xd, yd, prm, n, mud)
        ref = gp.loglik(xd, yd, kern, S2, RHO, TAU2, mu=mu, precision="fp64")
        out_ws = ref["out"].cpu().numpy()
        for k in range(3):  # loglik, logdet, q
            assert rel_err(out_na[k], out_ws[k]) < 1e-10, (n, k)
        assert rel_norm(alpha_na, ref["alpha"].cpu().numpy()) < 1e-10
        o = orc.loglik(x, y, kern, S2, RHO, TAU2, mu=mu)
        assert rel_err(out_na[0], o["loglik"]) < 1e-10, n
        assert rel_err(out_na[1], o["logdet"]) < 1e-10, n
        assert rel_err(out_na[2], o["quad"]) < 1e-10, n
        assert rel_norm(alpha_na, o["alpha"]) < 1e-10, n
    # above the static scratch: rejected up front
    n = NOALLOC_MAX_N + 1
    x = dev(inputs.uniform_points(n, 21999))
    y = dev(inputs.std_normal(n, 21998))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    prm = gp.params("exp", 1.0, 0.1, 0.1)
    st = L.gp_loglik_noalloc(gp._f64(x), gp._f64(y), None, n, ctypes.byref(prm), gp._f64(out),
                             None, gp._ptr(info), gp._stream())
    assert st == GP_ERR_TOO_LARGE
