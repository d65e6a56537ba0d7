"""Writes tests/golden/config4_n16384.npz: the oracle's log-likelihood,
log-determinant, quadratic form, gradient and alpha for the config-4 recipe
(Matern 5/2, theta = (0, log 0.05, log 0.1), uniform locations) at
n = 16,384, with y = L z formed from the oracle's own FP64 factor.

Only the oracle and the seeded input generators are called here; nothing
comes from the CUDA path.  Run from the repository root:
    python tests/golden/make_config4_golden.py [n]
(about 20 minutes on 8 cores at n = 16,384).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1305_4886_gb300 import inputs  # noqa: E402


def main(n=16384):
    oracle.build()
    p = inputs.config4(n)
    t0 = time.time()
    L = oracle.cholesky(oracle.cov_fill(p.x, p.kernel, p.s2, p.rho, p.tau2))
    y = oracle.lower_matvec(L, p.z)
    del L
    t1 = time.time()
    r = oracle.loglik_grad(p.x, y, p.kernel, p.s2, p.rho, p.tau2)
    t2 = time.time()
    path = os.path.join(HERE, f"config4_n{n}.npz")
    np.savez_compressed(path, n=n, y=y, loglik=r["loglik"], logdet=r["logdet"],
                        quad=r["quad"], grad=r["grad"], alpha=r["alpha"],
                        threads=oracle.num_threads(), seconds=np.array([t1 - t0, t2 - t1]))
    print(f"{path}: loglik {r['loglik']:.15g} grad {r['grad']} "
          f"({t1 - t0:.0f} s for y, {t2 - t1:.0f} s for loglik+grad, "
          f"{oracle.num_threads()} threads)")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 16384)
