"""The bounded dependency waits of the persistent batched launch.

A wait is made to run out on purpose, without any GPU fault: the testing aid
gp_batched_test_unset_tile makes every wait for one Cholesky tile of one
problem behave as if the tile were never produced, and a short wait limit
(gp_batched_set_wait_limit) ends that wait.  The FP64 form is used (CUDA
cores only: no tensor memory or bulk copies are in flight when CTAs leave).
Checked: the launch returns; that problem reports d_info = -1 and NaN
results; every other problem of the batch finished and matches the oracle;
and the next call on the same workspace succeeds (the device stays usable).
"""
import numpy as np
import pytest
import torch

from paper_1305_4886_gb300 import inputs
from tests.gpu_util import dev, rel_err, require_cuda

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_device_stays_usable(orc):
    require_cuda()
    from paper_1305_4886_gb300 import build, gp
    build.build()
    probs = inputs.config5(nprob=14, n_lo=64, n_hi=700)
    ys = [inputs.std_normal(p.n, 43000 + i) for i, p in enumerate(probs)]
    refs = [orc.loglik_grad(p.x, y, p.kernel, p.s2, p.rho, p.tau2) for p, y in zip(probs, ys)]
    xs, yd = [dev(p.x) for p in probs], [dev(y) for y in ys]
    prms = [gp.params(p.kernel, p.s2, p.rho, p.tau2) for p in probs]
    victim = int(np.argmax([p.n for p in probs]))
    T = -(-probs[victim].n // 64)  # FP64 form: 64 x 64 tiles
    assert T >= 3

    def check_clean(out, grad, info, skip):
        for i, ref in enumerate(refs):
            if i == skip:
                continue
            assert info[i] == 0, (i, info[i])
            assert rel_err(out[i, 0], ref["loglik"]) < 1e-10, i
            gerr = np.max(np.abs(grad[i] - ref["grad"])) / np.max(np.abs(ref["grad"]))
            assert gerr < 1e-9, (i, gerr)

    try:
        gp.gp_batched_set_wait_limit(0.25)
        gp.gp_batched_test_unset_tile(victim, T - 1, 0)
        r = gp.loglik_grad_batched(xs, yd, prms, precision="fp64")
        torch.cuda.synchronize()  # the launch returns: the wait ended at its limit
        info = r["info"].cpu().numpy()
        out, grad = r["out"].cpu().numpy(), r["grad"].cpu().numpy()
        assert info[victim] == -1, info
        assert np.all(np.isnan(out[victim])) and np.all(np.isnan(grad[victim]))
        check_clean(out, grad, info, victim)
    finally:
        gp.gp_batched_test_unset_tile(-1)
        gp.gp_batched_set_wait_limit(20.0)
    # the same workspace again, nothing left unset: every problem succeeds
    out = torch.full_like(r["out"], 7.0)
    grad = torch.full_like(r["grad"], 7.0)
    info = torch.full_like(r["info"], 99)
    gp.gp_loglik_grad_batched(r["batch"], "fp64", r["ws"], out, grad, info)
    torch.cuda.synchronize()
    check_clean(out.cpu().numpy(), grad.cpu().numpy(), info.cpu().numpy(), -1)
