"""torch.autograd.Function over gp_loglik_grad.

The forward pass evaluates the log-likelihood and its gradient with respect
to theta = (log sigma2, log rho, log tau2) in one call of the C ABI (the
gradient comes from the blocked Cholesky adjoint in libgp); the backward pass
only scales the stored gradient by the incoming one.  theta may live on any
device; locations and data must be float64 CUDA tensors.
"""
import torch

from . import gp


class GPLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, x, y, kernel, precision, mu, ws):
        th = theta.detach().to("cpu", torch.float64)
        s2, rho, tau2 = torch.exp(th).tolist()
        r = gp.loglik_grad(x, y, kernel, s2, rho, tau2, mu=mu, precision=precision, ws=ws,
                           want_alpha=False)
        ctx.save_for_backward(r["grad"].to(theta.device, theta.dtype))
        return r["out"][0].to(theta.device, theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None, None


def gp_marginal_loglik(theta, x, y, kernel="matern32", precision="mixed_f16", mu=None, ws=None):
    """Differentiable log-likelihood: theta = (log sigma2, log rho, log tau2).
    Pass a workspace from gp.workspace(n, precision, want_grad=True) to reuse
    device memory across calls."""
    return GPLogLik.apply(theta, x, y, kernel, precision, mu, ws)
