"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the method (no kernel evaluation, no
factorisation): it draws point locations, standard-normal vectors and
parameter values with numpy's PCG64 generator, so that both sides of every
parity test consume byte-identical arrays.

The workloads are synthetic stand-ins shaped like the paper's (Sec. 3 times
Cholesky factors of n = 32,768; the Sec. 4 supernova data set has
n = 67,275 = 25 spectra x 2691 wavelengths, which is not available).
Where a recipe needs y = L z with the FP64 factor L of C(theta), this module
returns z and the caller forms y with whichever factor its side owns.
"""
from dataclasses import dataclass, field

import numpy as np

KERNEL_IDS = {"exp": 0, "matern32": 1, "matern52": 2}


@dataclass
class Problem:
    name: str
    n: int
    kernel: str
    s2: float
    rho: float
    tau2: float
    x: np.ndarray                 # (n, 2) float64, interleaved coordinates
    mu: float = 0.0               # constant mean
    y: np.ndarray = None          # data vector when the recipe fixes it directly
    z: np.ndarray = None          # N(0,1) draws when y = L z
    meta: dict = field(default_factory=dict)

    @property
    def y_from_factor(self):
        return self.y is None


def uniform_points(n, seed):
    """n points uniform on [0,1]^2."""
    return np.random.default_rng(seed).random((n, 2))


def clustered_points(n, seed, n_centres=50, sd=0.02, frac_clustered=0.8):
    """Mixture of n_centres isotropic Gaussian clusters (centres uniform on
    [0,1]^2, standard deviation sd, no clipping) holding round(frac*n) points,
    plus a uniform background for the rest."""
    rng = np.random.default_rng(seed)
    centres = rng.random((n_centres, 2))
    m = int(round(frac_clustered * n))
    which = rng.integers(0, n_centres, size=m)
    pts_c = centres[which] + sd * rng.standard_normal((m, 2))
    pts_u = rng.random((n - m, 2))
    return np.concatenate([pts_c, pts_u], axis=0)


def std_normal(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


def exp_fill_1d(n, seed, spacing=0.01):
    """Sorted 1-D points (second coordinate 0) with random gaps; used for the
    exponential (Markov) covariance pins."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(spacing * (0.2 + rng.random(n)))
    return np.stack([t, np.zeros(n)], axis=1)


# ---------------------------------------------------------------------------
# The five workloads.  `n` may be overridden to get a smaller case with the
# same recipe (the parity tests run the oracle at sizes it finishes quickly).
# ---------------------------------------------------------------------------

def config1(n=1024):
    """Exponential, s2=1, rho=0.1, tau2=0.1, mu=0; y = L z, z ~ N(0,1)."""
    seed = 48861
    return Problem("exp-n%d-uniform" % n, n, "exp", 1.0, 0.1, 0.1,
                   uniform_points(n, seed), 0.0, None, std_normal(n, seed + 100))


def config2(n=16384):
    """Matern 3/2, s2=1, rho=0.05, tau2=0.05, mu=0.5;
    y = sin(6 x1) cos(4 x2) + N(0, 0.3^2)."""
    seed = 48862
    x = uniform_points(n, seed)
    noise = 0.3 * std_normal(n, seed + 100)
    y = np.sin(6.0 * x[:, 0]) * np.cos(4.0 * x[:, 1]) + noise
    return Problem("matern32-n%d-uniform" % n, n, "matern32", 1.0, 0.05, 0.05, x, 0.5, y, None)


def config3(n=67275):
    """Matern 3/2, s2=1, rho=0.02, tau2=0.1, mu=0 on 50 clusters (sd 0.02)
    plus 20% uniform background; y = L z."""
    seed = 48863
    return Problem("matern32-n%d-clustered" % n, n, "matern32", 1.0, 0.02, 0.1,
                   clustered_points(n, seed), 0.0, None, std_normal(n, seed + 100))


def config4(n=32768):
    """Matern 5/2, theta = (log s2, log rho, log tau2) = (0, log 0.05, log 0.1),
    mu = 0; y = L z."""
    seed = 48864
    return Problem("matern52-n%d-uniform" % n, n, "matern52", 1.0, 0.05, 0.1,
                   uniform_points(n, seed), 0.0, None, std_normal(n, seed + 100))


def config5(nprob=512, n_lo=256, n_hi=4096):
    """Independent problems: n log-uniform in [n_lo, n_hi]; exponential on
    even indices, Matern 3/2 on odd; rho ~ U[0.02, 0.3], s2 ~ U[0.5, 2],
    tau2 ~ U[0.01, 0.2]; uniform locations; y = L z per problem."""
    seed = 48865
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=nprob))).astype(np.int64)
    rho = rng.uniform(0.02, 0.3, size=nprob)
    s2 = rng.uniform(0.5, 2.0, size=nprob)
    tau2 = rng.uniform(0.01, 0.2, size=nprob)
    probs = []
    for i in range(nprob):
        n = int(ns[i])
        kern = "exp" if i % 2 == 0 else "matern32"
        x = np.random.default_rng([seed, i]).random((n, 2))
        z = np.random.default_rng([seed, i, 100]).standard_normal(n)
        probs.append(Problem("batch-%d" % i, n, kern, float(s2[i]), float(rho[i]),
                             float(tau2[i]), x, 0.0, None, z))
    return probs


def product_grid(n_t=25, n_w=2691, seed=48866):
    """The shape of the paper's example data set (Sec. 4.1: 25 spectra of a
    supernova at phases between -15 and 24 days, 2691 wavelengths each,
    n = 67,275), synthetic: phases sorted uniform in [-15, 24] days, log
    wavelengths on an even grid over [log 3500, log 7000] (angstrom), point
    (t, w) = (phase, log wavelength) phase-major; known measurement-error
    variances v_i uniform in [0.5e-5, 2e-5]; parameters at the maximum-
    likelihood values the paper reports for its fit (Sec. 4.3: sigma2 =
    0.0071, rho_t = 2.33, rho_w = 0.0089, tau2 = 2.6e-5); y = L z."""
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(-15.0, 24.0, size=n_t))
    w = np.linspace(np.log(3500.0), np.log(7000.0), n_w)
    x = np.stack([np.repeat(t, n_w), np.tile(w, n_t)], axis=1)
    n = n_t * n_w
    v = rng.uniform(0.5e-5, 2e-5, size=n)
    p = Problem("product-%dx%d" % (n_t, n_w), n, "product_matern2", 0.0071, 2.33, 2.6e-5, x, 0.0,
                None, np.random.default_rng(seed + 100).standard_normal(n))
    p.meta = {"rho_w": 0.0089, "v": v, "n_t": n_t, "n_w": n_w}
    return p
