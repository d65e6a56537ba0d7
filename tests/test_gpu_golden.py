"""Full parity against the oracle at n = 16,384 (the config-4 recipe: Matern
5/2, theta = (0, log 0.05, log 0.1), uniform locations, y = L z with the
oracle's FP64 factor).  The expected values (loglik, logdet, q, gradient,
alpha) and y were written by tests/golden/make_config4_golden.py, which
calls only the oracle.

Tolerances: the FP64 form and the FP64-grade form (five BF16 slices) at the
FP64 bar, 1e-10 relative on loglik and 1e-9 on the gradient (max norm) and
alpha (2-norm); the mixed form at its stated bound, 1e-6 on loglik and
gradient.
"""
import os

import numpy as np
import pytest

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import dev, rel_err, rel_norm, require_cuda

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config4_n16384.npz")


@pytest.fixture(scope="module")
def case():
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    ref = np.load(GOLDEN)
    n = int(ref["n"])
    p = inputs.config4(n)
    return gp, p, ref


@pytest.mark.parametrize("precision,tl,tg,ta", [("fp64", 1e-10, 1e-9, 1e-9),
                                                ("emu_fp64", 1e-10, 1e-9, 1e-9),
                                                ("mixed_f16", 1e-6, 1e-6, 1e-6)])
def test_config4_n16384_against_oracle(case, precision, tl, tg, ta):
    gp, p, ref = case
    r = gp.loglik_grad(dev(p.x), dev(ref["y"]), p.kernel, p.s2, p.rho, p.tau2,
                       precision=precision)
    out = r["out"].cpu().numpy()
    grad = r["grad"].cpu().numpy()
    assert rel_err(out[0], float(ref["loglik"])) < tl, (out[0], float(ref["loglik"]))
    assert rel_err(out[1], float(ref["logdet"])) < tl
    assert rel_err(out[2], float(ref["quad"])) < tl
    gerr = np.max(np.abs(grad - ref["grad"])) / np.max(np.abs(ref["grad"]))
    assert gerr < tg, (grad, ref["grad"], gerr)
    assert rel_norm(r["alpha"].cpu().numpy(), ref["alpha"]) < ta
