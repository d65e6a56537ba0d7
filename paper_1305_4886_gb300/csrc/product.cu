// product.cu -- the paper's example covariance (Sec. 4.2): the flux at
// phase t and log wavelength w is a Gaussian-process value plus a random
// effect of its phase plus measurement error of known variance v_i, so
//   C_ij = sigma2 k(|t_i - t_j| / rho_t) k(|w_i - w_j| / rho_w)
//          + tau2 [t_i == t_j] + v_i [i == j],
// a separable product of two Matern correlations of smoothness nu = 2, in the
// Rasmussen & Williams scaling a = sqrt(2 nu) u = 2u:
//   k(u) = a^2 K_2(a) / 2 (k(0) = 1),   -u k'(u) = a^3 K_1(a) / 2,
// the latter for the derivatives in log rho_t and log rho_w.
//
// Evaluation: both functions of a are tabulated once per process as
// piecewise Chebyshev series of degree 20, on 20 octaves [2^e, 2^(e+1)) for
// a in [2^-20, 1) (the functions carry a^4 log a terms at 0, analytic away
// from it) and on unit intervals up to a = 48 (beyond it k < 1e-18: 0).
// Below 2^-20 the two leading terms of the expansions at 0 are exact to the
// last bit.  The table is built on the host from the integral representation
//   K_nu(x) = exp(-x) int_0^inf exp(-2 x sinh^2(s/2)) cosh(nu s) ds
// (trapezoidal rule, geometric convergence for this
// integrand) and travels to the kernels as a kernel parameter (23 KB): no
// device memory, nothing to initialise per device.  One evaluation is a
// Clenshaw sum of 21 terms on the FP64 pipe.
//
// The fill, the matrix-free product C alpha of the refinement and the
// gradient contraction of this model run in FP64 in every precision form;
// the factorisation, solves and inverse are the common ones.
#include <math.h>

#include <mutex>

#include "internal.h"
#include "kern.cuh"

namespace gp {

constexpr int M2_NC = 21;               // Chebyshev coefficients per interval
constexpr int M2_OCT = 20;              // octaves below a = 1
constexpr int M2_AMAX = 48;             // k = 0 from here on
constexpr int M2_NI = 1 + M2_OCT + (M2_AMAX - 1);  // series, octaves, unit intervals

struct M2Tab {
    double c[2][M2_NI][M2_NC];  // [function][interval][coefficient], c0 pre-halved
};

// ---- host: the table ------------------------------------------------------
// K_nu(x) by the trapezoidal rule on the integral representation above, step
// min(1/32, 1/(8 sqrt(x))) (for large x the integrand is a peak of width
// about 1/sqrt(x)), terms summed with compensation until they vanish.
static double bessel_k_host(int nu, double x) {
    const double h = fmin(1.0 / 32.0, 0.125 / sqrt(x));
    double sum = 0.5, comp = 0.0;
    for (int k = 1; k < 400000; ++k) {
        const double t = h * k;
        const double sh = sinh(0.5 * t);
        const double e = 2.0 * x * sh * sh;
        const double term = exp(-e) * cosh(nu * t);
        const double y = term - comp, z = sum + y;
        comp = (z - sum) - y;
        sum = z;
        if (e > 50.0 && term < 1e-30 * sum) break;
    }
    return exp(-x) * h * sum;
}

// f = 0: a^2 K_2(a) / 2;  f = 1: a^3 K_1(a) / 2
static double m2_ref(int f, double a) {
    return f == 0 ? 0.5 * a * a * bessel_k_host(2, a) : 0.5 * a * a * a * bessel_k_host(1, a);
}

static void m2_interval(int idx, double &lo, double &hi) {
    if (idx <= M2_OCT) {  // octave [2^e, 2^(e+1)), e = idx - 21
        lo = ldexp(1.0, idx - 21);
        hi = 2.0 * lo;
    } else {
        lo = (double)(idx - M2_OCT);
        hi = lo + 1.0;
    }
}

// Chebyshev interpolants at the 21 Chebyshev points of each interval
// (coefficients by the discrete cosine sums, first one halved).
static const M2Tab &m2_table() {
    static M2Tab tab;
    static std::once_flag once;
    std::call_once(once, [] {
        const double PI = 3.141592653589793238462643383;
        for (int f = 0; f < 2; ++f) {
            for (int q = 0; q < M2_NC; ++q) tab.c[f][0][q] = 0.0;
            for (int idx = 1; idx < M2_NI; ++idx) {
                double lo, hi;
                m2_interval(idx, lo, hi);
                const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
                double fv[M2_NC];
                for (int k = 0; k < M2_NC; ++k)
                    fv[k] = m2_ref(f, mid + half * cos(PI * (k + 0.5) / M2_NC));
                for (int j = 0; j < M2_NC; ++j) {
                    long double s = 0.0L;
                    for (int k = 0; k < M2_NC; ++k)
                        s += (long double)fv[k] * (long double)cos(PI * j * (k + 0.5) / M2_NC);
                    s *= 2.0L / M2_NC;
                    if (j == 0) s *= 0.5L;
                    tab.c[f][idx][j] = (double)s;
                }
            }
        }
    });
    return tab;
}

// ---- device: evaluation ---------------------------------------------------
// f = 0: k(a) = a^2 K_2(a) / 2; f = 1: a^3 K_1(a) / 2, for a >= 0.
__device__ __forceinline__ double m2_eval(const M2Tab &T, int f, double a) {
    if (!(a < (double)M2_AMAX)) return 0.0;
    if (a < 0x1p-20) return f == 0 ? fma(-0.25 * a, a, 1.0) : 0.5 * a * a;
    int idx;
    double lo, hi;
    if (a < 1.0) {
        const int e = (int)((__double_as_longlong(a) >> 52) & 0x7FF) - 1023;  // a in [2^e, 2^(e+1))
        idx = e + 21;
        lo = __longlong_as_double((long long)(e + 1023) << 52);
        hi = 2.0 * lo;
    } else {
        const int j = (int)a;
        idx = M2_OCT + j;
        lo = (double)j;
        hi = lo + 1.0;
    }
    const double x = (2.0 * a - (lo + hi)) / (hi - lo);
    const double *c = T.c[f][idx];
    double b1 = 0.0, b2 = 0.0;
#pragma unroll
    for (int j = M2_NC - 1; j >= 1; --j) {
        const double b0 = fma(2.0 * x, b1, c[j] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(x, b1, c[0] - b2);
}

struct ProdPar {
    double s2, st, sw, tau2;  // st = 2 / rho_t, sw = 2 / rho_w
    const double *v;          // per-point variances (nullable)
};

// The phase factor k(|t_i - t_j| / rho_t) of the last pair a thread saw: rows
// and columns of a tile mostly share their phase (the data are phase by
// phase), so the factor is reused instead of re-evaluated.
struct PhaseMemo {
    double dt = -1.0, kt = 0.0, gt = 0.0;
};

__device__ __forceinline__ double prod_entry(const M2Tab &T, const ProdPar &p, double2 xi,
                                             double2 xj, PhaseMemo &m) {
    const double dt = fabs(xi.x - xj.x), dw = fabs(xi.y - xj.y);
    if (dt != m.dt) {
        m.dt = dt;
        m.kt = m2_eval(T, 0, dt * p.st);
    }
    double c = p.s2 * m.kt * m2_eval(T, 0, dw * p.sw);
    if (dt == 0.0) c += p.tau2;
    return c;
}

__device__ __forceinline__ double prod_diag(const ProdPar &p, int64_t i) {
    return p.s2 + p.tau2 + (p.v ? p.v[i] : 0.0);
}

// Lower 64 x 64 tiles of C (ld ldc), identity in the padding.
__global__ void __launch_bounds__(256) prod_fill_kernel(const double2 *__restrict__ x, int64_t n,
                                                        ProdPar p, const __grid_constant__ M2Tab T,
                                                        double *__restrict__ C, int64_t ldc,
                                                        int64_t *info) {
    __shared__ double2 xc[TB];
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    const int tid = threadIdx.x;
    if (tid < TB) {
        const int64_t j = col0 + tid;
        double2 q = make_double2(0.0, 0.0);
        if (j < n) {
            q = x[j];
            const double vj = p.v ? p.v[j] : 0.0;
            if (info && (!isfinite(q.x) || !isfinite(q.y) || !(vj >= 0.0) || !isfinite(vj)))
                set_info(info, -2);
        }
        xc[tid] = q;
    }
    __syncthreads();
    const int r = tid & (TB - 1), cg = tid >> 6;
    const int64_t i = row0 + r;
    const double2 xi = i < n ? x[i] : make_double2(0.0, 0.0);
    double *col = C + i;
    PhaseMemo memo;
    for (int c = cg; c < TB; c += 4) {
        const int64_t j = col0 + c;
        double v;
        if (i < n && j < n) v = (i == j) ? prod_diag(p, i) : prod_entry(T, p, xi, xc[c], memo);
        else v = (i == j) ? 1.0 : 0.0;
        col[j * ldc] = v;
    }
}

// acc += C a over one lower tile (each pair once, applied to both rows):
// row sums in registers, column sums by warp reductions (one lane writes each
// half-column partial), then one FP64 atomic per row and column.
__global__ void __launch_bounds__(256) prod_matvec_kernel(const double2 *__restrict__ x, int64_t n,
                                                          ProdPar p,
                                                          const __grid_constant__ M2Tab T,
                                                          const double *__restrict__ a,
                                                          double *acc, const int *skip,
                                                          const int64_t *info) {
    __shared__ double2 xc[TB];
    __shared__ double ac[TB];
    __shared__ double colpart[2][TB];
    if ((skip && *skip) || failed(info)) return;
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    if (row0 >= n) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int r = tid & (TB - 1), cg = tid >> 6, half = (tid >> 5) & 1;
    if (tid < TB) {
        const int64_t j = col0 + tid;
        xc[tid] = (j < n) ? x[j] : make_double2(0.0, 0.0);
        ac[tid] = (j < n) ? a[j] : 0.0;
    }
    __syncthreads();
    const int64_t i = row0 + r;
    const bool diag = ti == tj, row_ok = i < n;
    const double2 xi = row_ok ? x[i] : make_double2(0.0, 0.0);
    const double ai = row_ok ? a[i] : 0.0;
    double rs = 0.0;
    PhaseMemo memo;
    for (int c = cg; c < TB; c += 4) {
        const int64_t j = col0 + c;
        double cs = 0.0;
        // the diagonal tile: each pair once (j <= i)
        if (row_ok && j < n && !(diag && j > i)) {
            const double v = (i == j) ? prod_diag(p, i) : prod_entry(T, p, xi, xc[c], memo);
            rs = fma(v, ac[c], rs);
            if (i != j) cs = v * ai;  // C_ji a_i into row j
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        if (lane == 0) colpart[half][c] = cs;
    }
    if (row_ok) atomicAdd(acc + i, rs);
    __syncthreads();
    if (tid < TB) {
        const int64_t j = col0 + tid;
        const double cs = colpart[0][tid] + colpart[1][tid];
        if (j < n && cs != 0.0) atomicAdd(acc + j, cs);
    }
}

// Gradient shares of one lower tile of W = C^{-1} (ld), with alpha:
//   Cbar_ij = (a_i a_j - W_ij) / 2, off-diagonal pairs counted twice;
//   g = sum Cbar_ij dC_ij/dtheta, theta = (log s2, log rho_t, log rho_w, log tau2).
__global__ void __launch_bounds__(256) prod_grad_kernel(const double2 *__restrict__ x, int64_t n,
                                                        ProdPar p, const __grid_constant__ M2Tab T,
                                                        const double *W, int64_t ld,
                                                        const double *a, double *part,
                                                        const int64_t *info) {
    __shared__ double2 xc[TB];
    __shared__ double ac[TB];
    __shared__ double red[4][8];
    if (failed(info)) return;
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    const int tid = threadIdx.x;
    if (tid < TB) {
        const int64_t j = col0 + tid;
        xc[tid] = (j < n) ? x[j] : make_double2(0.0, 0.0);
        ac[tid] = (j < n) ? a[j] : 0.0;
    }
    __syncthreads();
    const int r = tid & (TB - 1), cg = tid >> 6;
    const int64_t i = row0 + r;
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    PhaseMemo memo;
    if (i < n) {
        const double2 xi = x[i];
        const double ai = a[i];
        for (int c = cg; c < TB; c += 4) {
            const int64_t k = col0 + c;
            if (k >= n || k > i) continue;
            const double w = W[i + k * ld];
            if (k == i) {
                const double cb = 0.5 * (ai * ai - w);
                g[0] = fma(cb, p.s2, g[0]);
                g[3] = fma(cb, p.tau2, g[3]);
            } else {
                const double cb2 = fma(ai, ac[c], -w);  // 2 Cbar_ik
                const double dt = fabs(xi.x - xc[c].x), dw = fabs(xi.y - xc[c].y);
                if (dt != memo.dt) {
                    memo.dt = dt;
                    memo.kt = m2_eval(T, 0, dt * p.st);
                    memo.gt = m2_eval(T, 1, dt * p.st);
                }
                const double aw = dw * p.sw;
                const double kt = memo.kt, kw = m2_eval(T, 0, aw);
                const double ks = p.s2 * cb2;
                g[0] = fma(ks * kt, kw, g[0]);
                g[1] = fma(ks * memo.gt, kw, g[1]);
                g[2] = fma(ks * kt, m2_eval(T, 1, aw), g[2]);
                if (dt == 0.0) g[3] = fma(cb2, p.tau2, g[3]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g[q] += __shfl_xor_sync(0xffffffffu, g[q], o);
    if ((tid & 31) == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[q][tid >> 5] = g[q];
    __syncthreads();
    if (tid < 4) {
        double s = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) s += red[tid][w8];
        part[4 * (int64_t)blockIdx.x + tid] = s;
    }
}

// grad[q] = compensated sum of the tiles' shares, in tile order.
__global__ void __launch_bounds__(1024) prod_grad_reduce_kernel(const double *part, int64_t ntiles,
                                                                double *grad,
                                                                const int64_t *info) {
    __shared__ double ps[4][1024];
    double s[4] = {0.0, 0.0, 0.0, 0.0}, c[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t t = threadIdx.x; t < ntiles; t += 1024)
        for (int q = 0; q < 4; ++q) {
            const double x = part[4 * t + q], u = s[q] + x;
            c[q] += (fabs(s[q]) >= fabs(x)) ? (s[q] - u) + x : (x - u) + s[q];
            s[q] = u;
        }
    for (int q = 0; q < 4; ++q) ps[q][threadIdx.x] = s[q] + c[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        double S = 0.0, Cc = 0.0;
        for (int t = 0; t < 1024; ++t) {
            const double x = ps[q][t], u = S + x;
            Cc += (fabs(S) >= fabs(x)) ? (S - u) + x : (x - u) + S;
            S = u;
        }
        grad[q] = (*info != 0) ? nan("") : S + Cc;
    }
}

static ProdPar prod_par(const KernParams &kp) {
    ProdPar p;
    p.s2 = kp.s2;
    p.st = kp.prod_st;
    p.sw = kp.prod_sw;
    p.tau2 = kp.tau2;
    p.v = kp.prod_v;
    return p;
}

int prod_fill(const double *d_x, int64_t n, int64_t np, const KernParams &kp, double *d_C,
              int64_t ldc, int64_t *d_info, cudaStream_t s) {
    const int64_t T = np / TB;
    const int ev = prof_start(s);
    prod_fill_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(
        reinterpret_cast<const double2 *>(d_x), n, prod_par(kp), m2_table(), d_C, ldc, d_info);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_FILL, 0.0, 8.0 * (double)np * (double)(np + 1) / 2.0);
    return GP_OK;
}

int prod_matvec(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *a,
                double *acc, const int *skip, const int64_t *info, cudaStream_t s) {
    const int64_t T = np / TB;
    prod_matvec_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(
        reinterpret_cast<const double2 *>(d_x), n, prod_par(kp), m2_table(), a, acc, skip, info);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

int prod_grad(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *W,
              int64_t ld, const double *alpha, double *part, double *grad, const int64_t *info,
              cudaStream_t s) {
    const int64_t T = np / TB, nt = T * (T + 1) / 2;
    const int ev = prof_start(s);
    prod_grad_kernel<<<(unsigned)nt, 256, 0, s>>>(reinterpret_cast<const double2 *>(d_x), n,
                                                   prod_par(kp), m2_table(), W, ld, alpha, part,
                                                   info);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_GRAD, 0.0, 8.0 * (double)np * (double)(np + 1) / 2.0);
    prod_grad_reduce_kernel<<<1, 1024, 0, s>>>(part, nt, grad, info);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

}  // namespace gp
