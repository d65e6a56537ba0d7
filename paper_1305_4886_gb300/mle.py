"""Maximum-likelihood fit of (sigma2, rho, tau2) with L-BFGS-B (Sec. 4.3
maximises the log-likelihood with L-BFGS-B; here the optimiser gets the
analytic gradient from gp_loglik_grad instead of finite differences).

The optimiser runs on the host (scipy); every function and gradient
evaluation is one gp_loglik_grad call on the device, reusing one workspace.
Evaluations at a theta already seen are served from a one-entry cache, like
the paper's "up-to-date" bookkeeping of computed objects (Sec. 2.3.4).
"""
import numpy as np
import torch

from . import gp


def fit(x, y, kernel="matern32", theta0=(0.0, np.log(0.1), np.log(0.1)), precision="mixed_f16",
        mu=None, bounds=((-10, 10), (-12, 5), (-20, 5)), maxiter=60, tol=1e-9):
    """x: (n, 2) float64 CUDA tensor, y: (n,) float64 CUDA tensor.  Returns a
    dict with theta (log parameters), params (natural), loglik, grad, nfev,
    success and message."""
    from scipy.optimize import minimize

    n = x.shape[0]
    ws = gp.workspace(n, precision, want_grad=True, device=x.device)
    cache = {}
    count = {"n": 0}

    def evaluate(th):
        key = tuple(np.round(np.asarray(th, dtype=np.float64), 15))
        if key not in cache:
            s2, rho, tau2 = np.exp(th)
            r = gp.loglik_grad(x, y, kernel, s2, rho, tau2, mu=mu, precision=precision, ws=ws,
                               want_alpha=False)
            cache.clear()
            cache[key] = (float(r["out"][0]), r["grad"].cpu().numpy().copy())
            count["n"] += 1
        return cache[key]

    def f(th):
        v, _ = evaluate(th)
        return -v

    def g(th):
        _, gr = evaluate(th)
        return -gr

    res = minimize(f, np.asarray(theta0, dtype=np.float64), jac=g, method="L-BFGS-B",
                   bounds=bounds, options={"maxiter": maxiter, "gtol": tol, "ftol": 1e-15})
    ll, gr = evaluate(res.x)
    return {"theta": res.x, "params": np.exp(res.x), "loglik": ll, "grad": gr,
            "nfev": count["n"], "success": bool(res.success), "message": str(res.message)}
