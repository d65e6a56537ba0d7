// kern.cuh -- covariance functions evaluated on the device (FP64).
//
// Sec. 1 of the paper: C(theta) = C_g(theta) + C_y(theta); the latent
// covariance is sigma2 * k(d / rho) and C_y = tau2 I (the nugget).  The
// Matern forms use the Rasmussen & Williams scaling a = sqrt(2 nu) d / rho.
// The same routine feeds the fill, the matrix-free residual and the
// gradient contraction, so that dC/dtheta is recomputed tile by tile and
// never stored.
//
// exp(-a) is evaluated with a table-driven reduction (Tang's method, 1989):
// with k = round(64 a / ln 2) = 64 m + j and r = a - k ln2/64 (|r| <= ln2/128,
// formed with a two-part ln2/64 so that k * hi is exact),
//     exp(-a) = 2^-m * 2^(-j/64) * exp(-r),
// exp(-r) by its degree-5 Taylor polynomial (truncation below 4e-17
// relative) and 2^(-j/64) from a 64-entry table computed on the host in
// extended precision.  About ten FP64 operations, which matters on a part
// whose FP64 pipe is 1/64 of its FP32 pipe; the kernels stage the table in
// shared memory.
#pragma once

#include <math.h>

#include "common.cuh"
#include "kern_df.cuh"

namespace gp {

constexpr int EXP_TAB = 64;

struct KernParams {
    int kind;        // gp_kernel
    double s2;       // sigma2
    double scale;    // multiplier turning d into the exponent argument a
    double diag;     // sigma2 + tau2
    double tau2;
    double tab[EXP_TAB];  // 2^(-j/64)
    int use_df;           // evaluate off-diagonal entries in double-float (FP32 pipe)
    KernDf kd;
    // the product model of product.cu (its fill, C alpha and gradient replace
    // the ones above): scales 2 / rho_t, 2 / rho_w and the per-point variances
    int product = 0;
    double prod_st = 0.0, prod_sw = 0.0;
    const double *prod_v = nullptr;
};

// use_df: the tensor-core forms, whose operand slices carry 2^-32 of the row
// bounds, take the double-float evaluation; the FP64 form stays in FP64.
inline KernParams make_kern(const gp_params &p, bool use_df = false) {
    KernParams k;
    k.use_df = use_df ? 1 : 0;
    k.kd = make_kern_df(p);
    k.kind = p.kernel;
    k.s2 = p.sigma2;
    double c = 1.0;
    if (p.kernel == GP_KERNEL_MATERN32) c = 1.7320508075688772;  // sqrt(3)
    if (p.kernel == GP_KERNEL_MATERN52) c = 2.2360679774997897;  // sqrt(5)
    k.scale = c / p.rho;
    k.diag = p.sigma2 + p.tau2;
    k.tau2 = p.tau2;
    for (int j = 0; j < EXP_TAB; ++j)
        k.tab[j] = static_cast<double>(exp2l(-static_cast<long double>(j) / EXP_TAB));
    return k;
}

// exp(-a) for a >= 0; tab = 2^(-j/64) in shared memory.
__device__ __forceinline__ double exp_neg(double a, const double *tab) {
    constexpr double INV_L = 92.33248261689366;           // 64 / ln 2
    constexpr double L_HI = 0.010830424696223417;         // ln2/64, 36 significant bits
    constexpr double L_LO = 2.572804622327669e-14;        // ln2/64 - L_HI
    constexpr double SHIFT = 6755399441055744.0;          // 1.5 * 2^52: round to integer
    if (!(a < 700.0)) return 0.0;                         // below 1e-304 (or NaN input)
    const double t = fma(a, INV_L, SHIFT);
    const int k = __double2loint(t);
    const double kd = t - SHIFT;
    double r = fma(-kd, L_HI, a);
    r = fma(-kd, L_LO, r);
    // exp(-r), |r| <= ln2/128
    double p = -1.0 / 120.0;
    p = fma(p, r, 1.0 / 24.0);
    p = fma(p, r, -1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, -1.0);
    p = fma(p, r, 1.0);
    double v = tab[k & (EXP_TAB - 1)] * p;
    // scale by 2^-m, m = k / 64 (k >= 0), on the exponent field
    const int m = k >> 6;
    const long long bits = __double_as_longlong(v) - (static_cast<long long>(m) << 52);
    return __longlong_as_double(bits);
}

// sigma2 * k(d / rho) for a distinct pair at distance d (scale = sqrt(2 nu) / rho).
__device__ __forceinline__ double cov_offdiag_s(int kind, double s2, double scale, double d,
                                                const double *tab) {
    const double a = d * scale;
    const double e = exp_neg(a, tab);
    if (kind == GP_KERNEL_EXP) return s2 * e;
    if (kind == GP_KERNEL_MATERN32) return s2 * fma(a, e, e);
    return s2 * (1.0 + a + a * a * (1.0 / 3.0)) * e;
}

__device__ __forceinline__ double cov_offdiag(const KernParams &k, double d, const double *tab) {
    return cov_offdiag_s(k.kind, k.s2, k.scale, d, tab);
}

// Off-diagonal entry and its derivative in log rho, -sigma2 u k'(u):
//   exp: s2 a e^-a;  Matern 3/2: s2 a^2 e^-a;  Matern 5/2: s2 a^2 (1+a)/3 e^-a.
__device__ __forceinline__ void cov_and_dlogrho_s(int kind, double s2, double scale, double d,
                                                  double &c, double &dr, const double *tab) {
    const double a = d * scale;
    const double e = exp_neg(a, tab);
    if (kind == GP_KERNEL_EXP) {
        c = s2 * e;
        dr = c * a;
    } else if (kind == GP_KERNEL_MATERN32) {
        c = s2 * fma(a, e, e);
        dr = s2 * a * a * e;
    } else {
        const double p = 1.0 + a;
        c = s2 * (p + a * a * (1.0 / 3.0)) * e;
        dr = s2 * a * a * p * (1.0 / 3.0) * e;
    }
}

__device__ __forceinline__ void cov_and_dlogrho(const KernParams &k, double d, double &c,
                                                double &dr, const double *tab) {
    cov_and_dlogrho_s(k.kind, k.s2, k.scale, d, c, dr, tab);
}

__device__ __forceinline__ double pair_dist(double2 p, double2 q) {
    const double dx = p.x - q.x, dy = p.y - q.y;
    return sqrt(dx * dx + dy * dy);
}

// Copy the exp table to shared memory (call before the CTA's first barrier).
__device__ __forceinline__ void stage_exp_table(const KernParams &k, double *tab) {
    if (threadIdx.x < EXP_TAB) tab[threadIdx.x] = k.tab[threadIdx.x];
}

}  // namespace gp
