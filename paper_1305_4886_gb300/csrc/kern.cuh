// kern.cuh -- covariance functions evaluated on the device (FP64).
//
// Sec. 1 of the paper: C(theta) = C_g(theta) + C_y(theta); the latent
// covariance is sigma2 * k(d / rho) and C_y = tau2 I (the nugget).  The
// Matern forms use the Rasmussen & Williams scaling a = sqrt(2 nu) d / rho.
// The same routine feeds the fill, the matrix-free residual and the
// gradient contraction, so that dC/dtheta is recomputed tile by tile and
// never stored.
#pragma once

#include "common.cuh"

namespace gp {

struct KernParams {
    int kind;        // gp_kernel
    double s2;       // sigma2
    double scale;    // multiplier turning d into the exponent argument a
    double diag;     // sigma2 + tau2
    double tau2;
};

inline KernParams make_kern(const gp_params &p) {
    KernParams k;
    k.kind = p.kernel;
    k.s2 = p.sigma2;
    double c = 1.0;
    if (p.kernel == GP_KERNEL_MATERN32) c = 1.7320508075688772;  // sqrt(3)
    if (p.kernel == GP_KERNEL_MATERN52) c = 2.2360679774997897;  // sqrt(5)
    k.scale = c / p.rho;
    k.diag = p.sigma2 + p.tau2;
    k.tau2 = p.tau2;
    return k;
}

// sigma2 * k(d / rho) for a distinct pair at distance d.
__device__ __forceinline__ double cov_offdiag(const KernParams &k, double d) {
    double a = d * k.scale;
    double e = exp(-a);
    if (k.kind == GP_KERNEL_EXP) return k.s2 * e;
    if (k.kind == GP_KERNEL_MATERN32) return k.s2 * fma(a, e, e);
    return k.s2 * (1.0 + a + a * a * (1.0 / 3.0)) * e;
}

// Off-diagonal entry and its derivative in log rho, -sigma2 u k'(u):
//   exp: s2 a e^-a;  Matern 3/2: s2 a^2 e^-a;  Matern 5/2: s2 a^2 (1+a)/3 e^-a.
__device__ __forceinline__ void cov_and_dlogrho(const KernParams &k, double d, double &c,
                                                double &dr) {
    double a = d * k.scale;
    double e = exp(-a);
    if (k.kind == GP_KERNEL_EXP) {
        c = k.s2 * e;
        dr = c * a;
    } else if (k.kind == GP_KERNEL_MATERN32) {
        c = k.s2 * fma(a, e, e);
        dr = k.s2 * a * a * e;
    } else {
        double p = 1.0 + a;
        c = k.s2 * (p + a * a * (1.0 / 3.0)) * e;
        dr = k.s2 * a * a * p * (1.0 / 3.0) * e;
    }
}

__device__ __forceinline__ double pair_dist(double2 p, double2 q) {
    double dx = p.x - q.x, dy = p.y - q.y;
    return sqrt(dx * dx + dy * dy);
}

}  // namespace gp
