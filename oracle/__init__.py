"""FP64 CPU oracle for the GP marginal log-likelihood (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product path never does.
"""
from .gp_oracle import (  # noqa: F401
    build,
    cov_fill,
    cov_rows,
    dcov_dlogrho,
    cholesky,
    forward,
    backward,
    lower_matvec,
    lower_inverse,
    inverse_from_chol,
    logdet,
    loglik,
    loglik_grad,
    kernel,
    kernel_dlogrho,
    num_threads,
    set_threads,
    cross_cov,
    predict,
    predict_from_data,
    bessel_k,
    matern2,
    matern2_dlogrho,
    prod_cov_fill,
    prod_loglik_grad,
    philox4x64,
    normals,
    simulate,
    simulate_conditional,
    OracleNotPD,
    KERNELS,
)
