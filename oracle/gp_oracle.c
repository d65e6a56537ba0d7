/*
 * gp_oracle.c -- plain, slow FP64 CPU oracle for the Gaussian-process
 * marginal log-likelihood of Paciorek et al., "Parallelizing Gaussian
 * Process Calculations in R" (arXiv:1305.4886).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this
 * code: only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header, table or helper
 * with the CUDA library; the two meet only through seeded inputs.
 *
 * What it computes, step by step, is the definition in Section 1 of the
 * paper, written out with unblocked loops:
 *
 *   marginal model      Y | theta ~ N(mu, C),  C = C_y + C_g      (Sec. 1)
 *   covariance entries  C_ij = s2 * k(d_ij / rho)   (i != j)
 *                       C_ii = s2 + tau2            (nugget, diagonal C_y)
 *   Cholesky            L L^T = C, no pivoting; a pivot <= 0 fails (Sec. 5)
 *   forward solve       v = L^{-1} (y - mu)          ("backsolve", Sec. 1)
 *   sum of squares      q = v^T v                    (Sec. 2.2.2)
 *   log-determinant     logdet = 2 sum_i log L_ii    (Sec. 2.2.2)
 *   log-density         l = -logdet/2 - q/2 - (n/2) log(2 pi)
 *
 * The paper writes the density only up to proportionality; the oracle keeps
 * the Gaussian normalising constant so that l is the full log-density.
 *
 * The gradient is not in the paper.  It is the standard Gaussian identity
 *   dl/dtheta_j = 1/2 alpha^T (dC/dtheta_j) alpha - 1/2 tr(C^{-1} dC/dtheta_j),
 *   alpha = C^{-1}(y - mu),
 * with theta = (log s2, log rho, log tau2), C^{-1} formed explicitly from the
 * inverse of L, and every trace / quadratic form summed over all (i, j).
 *
 * Kernels (Matern in the Rasmussen & Williams parameterisation, the paper's
 * GP reference; u = d / rho):
 *   exponential  k(u) = exp(-u)
 *   Matern 3/2   k(u) = (1 + a) exp(-a),            a = sqrt(3) u
 *   Matern 5/2   k(u) = (1 + a + a^2/3) exp(-a),    a = sqrt(5) u
 *
 * Storage: every matrix here is a full n x n row-major array (A[i*n + j]).
 * Locations are n points of 2 coordinates, interleaved (x_i1, x_i2).
 * Sums that feed the reported scalars use Neumaier compensation.
 * OpenMP parallelises independent rows only; each row's arithmetic is
 * sequential and rows are combined in index order, so results do not depend
 * on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_NOT_PD 1
#define ORC_INVALID 2

typedef struct {
    double s, c;
} nsum_t; /* Neumaier running sum */

static void ns_init(nsum_t *a) { a->s = 0.0; a->c = 0.0; }
static void ns_add(nsum_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double ns_get(const nsum_t *a) { return a->s + a->c; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* correlation k(u) for u = d/rho >= 0 (Sec. 1 covariance; kernels above) */
double orc_kernel(int kind, double u) {
    if (kind == 0) return exp(-u);
    if (kind == 1) {
        double a = sqrt(3.0) * u;
        return (1.0 + a) * exp(-a);
    }
    if (kind == 2) {
        double a = sqrt(5.0) * u;
        return (1.0 + a + a * a / 3.0) * exp(-a);
    }
    return NAN;
}

/* -u k'(u): derivative of k(d/rho) with respect to log rho */
double orc_kernel_dlogrho(int kind, double u) {
    if (kind == 0) return u * exp(-u);
    if (kind == 1) {
        double a = sqrt(3.0) * u;
        return a * a * exp(-a);
    }
    if (kind == 2) {
        double a = sqrt(5.0) * u;
        return a * a * (1.0 + a) / 3.0 * exp(-a);
    }
    return NAN;
}

static double dist2d(const double *x, int64_t i, int64_t j) {
    double dx = x[2 * i] - x[2 * j];
    double dy = x[2 * i + 1] - x[2 * j + 1];
    return sqrt(dx * dx + dy * dy);
}

/* C(theta): full symmetric n x n (Sec. 1: C = C_g + C_y, C_y = tau2 I) */
void orc_cov_fill(const double *x, int64_t n, int kind, double s2, double rho,
                  double tau2, double *C) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (i == j) C[i * n + j] = s2 + tau2;
            else C[i * n + j] = s2 * orc_kernel(kind, dist2d(x, i, j) / rho);
        }
    }
}

/* Selected rows of C(theta): out[r * n + j] = C[rows[r], j] (same definition
 * as orc_cov_fill), for checks at sizes where the full matrix is too big. */
void orc_cov_rows(const double *x, int64_t n, const int64_t *rows, int64_t nrows, int kind,
                  double s2, double rho, double tau2, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        for (int64_t j = 0; j < n; ++j) {
            if (i == j) out[r * n + j] = s2 + tau2;
            else out[r * n + j] = s2 * orc_kernel(kind, dist2d(x, i, j) / rho);
        }
    }
}

/* dC/dlog(rho): full symmetric, zero diagonal */
void orc_dcov_dlogrho(const double *x, int64_t n, int kind, double s2, double rho,
                      double *D) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (i == j) D[i * n + j] = 0.0;
            else D[i * n + j] = s2 * orc_kernel_dlogrho(kind, dist2d(x, i, j) / rho);
        }
    }
}

/* Unblocked column Cholesky, in place; lower triangle of A becomes L, the
 * strict upper triangle is zeroed.  No pivoting: returns j+1 for the first
 * column j whose pivot is not > 0 (the failure mode noted in Sec. 5). */
int64_t orc_cholesky(double *A, int64_t n) {
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return j + 1;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            const double *li = A + i * n, *lj = A + j * n;
            for (int64_t k = 0; k < j; ++k) t -= li[k] * lj[k];
            A[i * n + j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
    return 0;
}

/* v = L^{-1} b (forward substitution) */
void orc_forward(const double *L, int64_t n, const double *b, double *v) {
    for (int64_t i = 0; i < n; ++i) {
        double t = b[i];
        for (int64_t k = 0; k < i; ++k) t -= L[i * n + k] * v[k];
        v[i] = t / L[i * n + i];
    }
}

/* a = L^{-T} v (back substitution, column-oriented) */
void orc_backward(const double *L, int64_t n, const double *v, double *a) {
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(w, v, sizeof(double) * (size_t)n);
    for (int64_t i = n - 1; i >= 0; --i) {
        a[i] = w[i] / L[i * n + i];
        for (int64_t k = 0; k < i; ++k) w[k] -= L[i * n + k] * a[i];
    }
    free(w);
}

/* L * z (lower triangular times vector), used to draw y = L z */
void orc_lower_matvec(const double *L, int64_t n, const double *z, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t = 0.0;
        for (int64_t k = 0; k <= i; ++k) t += L[i * n + k] * z[k];
        y[i] = t;
    }
}

/* logdet = 2 sum log L_ii (Sec. 2.2.2), compensated */
double orc_logdet(const double *L, int64_t n) {
    nsum_t a;
    ns_init(&a);
    for (int64_t i = 0; i < n; ++i) ns_add(&a, log(L[i * n + i]));
    return 2.0 * ns_get(&a);
}

/* compensated inner product */
double orc_dot(const double *a, const double *b, int64_t n) {
    nsum_t s;
    ns_init(&s);
    for (int64_t i = 0; i < n; ++i) ns_add(&s, a[i] * b[i]);
    return ns_get(&s);
}

/* X = L^{-1}, by forward substitution on each unit vector; full row-major */
void orc_lower_inverse(const double *L, int64_t n, double *X) {
    memset(X, 0, sizeof(double) * (size_t)n * (size_t)n);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < n; ++c) {
        /* column c of X solves L x = e_c; x_i = 0 for i < c */
        for (int64_t i = c; i < n; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int64_t k = c; k < i; ++k) t -= L[i * n + k] * X[k * n + c];
            X[i * n + c] = t / L[i * n + i];
        }
    }
}

/* W = C^{-1} = L^{-T} L^{-1}, full symmetric */
void orc_inverse_from_chol(const double *L, int64_t n, double *W) {
    double *X = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double *XT = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    orc_lower_inverse(L, n, X);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = 0; k < n; ++k) XT[i * n + k] = X[k * n + i];
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            /* W_ij = sum_k X_ki X_kj, nonzero only for k >= max(i, j) = i */
            double t = 0.0;
            for (int64_t k = i; k < n; ++k) t += XT[i * n + k] * XT[j * n + k];
            W[i * n + j] = t;
            W[j * n + i] = t;
        }
    }
    free(X);
    free(XT);
}

static int params_ok(int64_t n, int kind, double s2, double rho, double tau2) {
    if (n < 1) return 0;
    if (kind < 0 || kind > 2) return 0;
    if (!(s2 > 0.0) || !(rho > 0.0) || !(tau2 >= 0.0)) return 0;
    if (!isfinite(s2) || !isfinite(rho) || !isfinite(tau2)) return 0;
    return 1;
}

/*
 * Log-likelihood (Sec. 1 / Sec. 2.2.2).  mu may be NULL (zero mean).
 * out[0] = loglik, out[1] = logdet, out[2] = q.  alpha (n, may be NULL)
 * receives C^{-1}(y - mu).  L (n*n, may be NULL) receives the factor.
 * Returns ORC_OK, ORC_INVALID, or ORC_NOT_PD (then *info = failing col + 1).
 */
int orc_loglik(const double *x, const double *y, const double *mu, int64_t n,
               int kind, double s2, double rho, double tau2, double *out,
               double *alpha, double *Lout, int64_t *info) {
    if (info) *info = 0;
    if (!params_ok(n, kind, s2, rho, tau2)) return ORC_INVALID;
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!isfinite(x[i])) return ORC_INVALID;
    size_t nn = (size_t)n * (size_t)n;
    double *C = (double *)malloc(sizeof(double) * nn);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    orc_cov_fill(x, n, kind, s2, rho, tau2, C);
    int64_t f = orc_cholesky(C, n);
    if (f != 0) {
        if (info) *info = f;
        out[0] = out[1] = out[2] = NAN;
        free(C); free(r); free(v);
        return ORC_NOT_PD;
    }
    for (int64_t i = 0; i < n; ++i) r[i] = y[i] - (mu ? mu[i] : 0.0);
    orc_forward(C, n, r, v);
    double logdet = orc_logdet(C, n);
    double q = orc_dot(v, v, n);
    out[0] = -0.5 * logdet - 0.5 * q - 0.5 * (double)n * log(2.0 * M_PI);
    out[1] = logdet;
    out[2] = q;
    if (alpha) orc_backward(C, n, v, alpha);
    if (Lout) memcpy(Lout, C, sizeof(double) * nn);
    free(C); free(r); free(v);
    return ORC_OK;
}

/*
 * Log-likelihood and its gradient with respect to
 * theta = (log s2, log rho, log tau2):
 *   dC/dlog s2  = C - tau2 I
 *   dC/dlog rho = s2 * (-u k'(u)),  u = d/rho  (zero on the diagonal)
 *   dC/dlog tau2 = tau2 I
 *   g_j = 1/2 alpha^T dC_j alpha - 1/2 sum_{i,k} W_ik (dC_j)_ik,  W = C^{-1}
 * Every sum runs over the full square with Neumaier compensation.
 */
int orc_loglik_grad(const double *x, const double *y, const double *mu, int64_t n,
                    int kind, double s2, double rho, double tau2, double *out,
                    double *alpha, double *grad, int64_t *info) {
    size_t nn = (size_t)n * (size_t)n;
    double *L, *W, *C, *D, *a;
    int st;
    if (!params_ok(n, kind, s2, rho, tau2)) return ORC_INVALID;
    L = (double *)malloc(sizeof(double) * nn);
    a = (double *)malloc(sizeof(double) * (size_t)n);
    st = orc_loglik(x, y, mu, n, kind, s2, rho, tau2, out, a, L, info);
    if (st != ORC_OK) {
        grad[0] = grad[1] = grad[2] = NAN;
        free(L); free(a);
        return st;
    }
    W = (double *)malloc(sizeof(double) * nn);
    C = (double *)malloc(sizeof(double) * nn);
    D = (double *)malloc(sizeof(double) * nn);
    orc_inverse_from_chol(L, n, W);
    orc_cov_fill(x, n, kind, s2, rho, tau2, C);
    orc_dcov_dlogrho(x, n, kind, s2, rho, D);

    /* per-row compensated partial sums, combined in row order */
    double *part = (double *)calloc((size_t)n * 6, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        nsum_t q0, q1, t0, t1;
        ns_init(&q0); ns_init(&q1); ns_init(&t0); ns_init(&t1);
        for (int64_t k = 0; k < n; ++k) {
            double dc0 = C[i * n + k] - (i == k ? tau2 : 0.0);
            double dc1 = D[i * n + k];
            ns_add(&q0, a[i] * dc0 * a[k]);
            ns_add(&q1, a[i] * dc1 * a[k]);
            ns_add(&t0, W[i * n + k] * dc0);
            ns_add(&t1, W[i * n + k] * dc1);
        }
        part[6 * i + 0] = ns_get(&q0);
        part[6 * i + 1] = ns_get(&q1);
        part[6 * i + 2] = ns_get(&t0);
        part[6 * i + 3] = ns_get(&t1);
        part[6 * i + 4] = a[i] * a[i];      /* alpha^T alpha term */
        part[6 * i + 5] = W[i * n + i];     /* tr W term */
    }
    nsum_t s[6];
    for (int c = 0; c < 6; ++c) ns_init(&s[c]);
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 6; ++c) ns_add(&s[c], part[6 * i + c]);
    grad[0] = 0.5 * ns_get(&s[0]) - 0.5 * ns_get(&s[2]);
    grad[1] = 0.5 * ns_get(&s[1]) - 0.5 * ns_get(&s[3]);
    grad[2] = 0.5 * tau2 * ns_get(&s[4]) - 0.5 * tau2 * ns_get(&s[5]);
    if (alpha) memcpy(alpha, a, sizeof(double) * (size_t)n);
    free(part); free(L); free(W); free(C); free(D); free(a);
    return ORC_OK;
}

/*
 * Kriging prediction (Sec. 1: prediction at new locations is the conditional
 * expectation of the latent process given the data, with its variance;
 * Sec. 2.2.2: it reuses the Cholesky factor through forward and back
 * solves; Sec. 4.3: predictions with standard errors on a grid).  For new
 * locations xs_1..xs_m (latent process Z, so no nugget between a new and a
 * training point):
 *   cross covariance  K_ij = s2 k(|x_i - xs_j| / rho)            (n x m)
 *   mean              m_j  = mu_new + sum_i K_ij alpha_i,  alpha = C^{-1}(y - mu)
 *   variance          v_j  = s2 - w_j^T w_j,  w_j = L^{-1} K_.j,
 * i.e. s2 - K_.j^T C^{-1} K_.j, the Schur complement of C in the joint
 * covariance of (Y, Z(xs_j)).
 */
static double dist2d_pair(const double *x, int64_t i, const double *xs, int64_t j) {
    double dx = x[2 * i] - xs[2 * j];
    double dy = x[2 * i + 1] - xs[2 * j + 1];
    return sqrt(dx * dx + dy * dy);
}

/* K (n x m, row-major): K[i * m + j] = s2 k(|x_i - xs_j| / rho) */
void orc_cross_cov(const double *x, int64_t n, const double *xs, int64_t m, int kind, double s2,
                   double rho, double *K) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j)
            K[i * m + j] = s2 * orc_kernel(kind, dist2d_pair(x, i, xs, j) / rho);
}

/*
 * mean (m) and, when var is not NULL, variance (m) at the new locations,
 * given the factor L (n x n row-major, lower) and alpha = C^{-1}(y - mu) of
 * the training data.  Each new location is independent of the others.
 */
void orc_predict(const double *x, int64_t n, const double *xs, int64_t m, int kind, double s2,
                 double rho, const double *L, const double *alpha, double mu_new, double *mean,
                 double *var) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        double *k = (double *)malloc(sizeof(double) * (size_t)n);
        double *w = (double *)malloc(sizeof(double) * (size_t)n);
        nsum_t s;
        ns_init(&s);
        for (int64_t i = 0; i < n; ++i) {
            k[i] = s2 * orc_kernel(kind, dist2d_pair(x, i, xs, j) / rho);
            ns_add(&s, k[i] * alpha[i]);
        }
        mean[j] = mu_new + ns_get(&s);
        if (var) {
            orc_forward(L, n, k, w);
            var[j] = s2 - orc_dot(w, w, n);
        }
        free(k);
        free(w);
    }
}

/*
 * Simulation (Sec. 1: unconditional realisations and realisations
 * conditional on the data; Sec. 2.3.2: multiplication of the Cholesky factor
 * by a matrix of standard normals; Sec. 4.3: 1000 posterior realisations).
 *
 * Random numbers come from the counter-based generator Philox4x64-10
 * (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC 2011): ten rounds on a 4 x 64-bit counter with a 2 x 64-bit
 * key; each round multiplies words 0 and 2 by the round constants, keeps
 * the high and low halves, and mixes in the other words and the key, which
 * is bumped by the Weyl constants between rounds.  The paper's package uses
 * another parallel generator (L'Ecuyer's, through rlecuyer); the draws
 * here are defined by this generator instead:
 *   for realisation c (0-based, offset by `first`) and rows 4q .. 4q+3,
 *   (w0, w1, w2, w3) = philox(counter = (q, first + c, stream, 0),
 *                             key = (seed, 0)),
 *   u_k = ((w_k >> 11) + 1/2) 2^-53, in (0, 1),
 *   z_{4q} = s0 cos(2 pi u1),  z_{4q+1} = s0 sin(2 pi u1),  s0 = sqrt(-2 ln u0),
 *   z_{4q+2} = s2 cos(2 pi u3), z_{4q+3} = s2 sin(2 pi u3), s2 = sqrt(-2 ln u2)
 * (the Box-Muller transform).
 */
void orc_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        const unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        const unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        const uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double u01(uint64_t w) { return ((double)(w >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/* out[c * n + i] = z_i of realisation first + c, i < n, c < r */
void orc_normals(int64_t n, int64_t r, uint64_t seed, uint64_t stream, uint64_t first, double *out) {
    const double TWO_PI = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < r; ++c) {
        for (int64_t q = 0; 4 * q < n; ++q) {
            uint64_t ctr[4] = {(uint64_t)q, first + (uint64_t)c, stream, 0};
            uint64_t key[2] = {seed, 0};
            uint64_t w[4];
            double z[4];
            orc_philox4x64(ctr, key, w);
            const double s0 = sqrt(-2.0 * log(u01(w[0]))), s2 = sqrt(-2.0 * log(u01(w[2])));
            z[0] = s0 * cos(TWO_PI * u01(w[1]));
            z[1] = s0 * sin(TWO_PI * u01(w[1]));
            z[2] = s2 * cos(TWO_PI * u01(w[3]));
            z[3] = s2 * sin(TWO_PI * u01(w[3]));
            for (int k = 0; k < 4 && 4 * q + k < n; ++k) out[c * n + 4 * q + k] = z[k];
        }
    }
}

/* Unconditional realisations: out[c * n + i] = mu + (L e_c)_i, e_c the normals
 * of realisation first + c (stream 0).  L: n x n row-major lower factor. */
void orc_simulate(const double *L, int64_t n, int64_t r, uint64_t seed, uint64_t first, double mu,
                  double *out) {
    double *E = (double *)malloc(sizeof(double) * (size_t)n * (size_t)r);
    orc_normals(n, r, seed, 0, first, E);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < r; ++c) {
        for (int64_t i = 0; i < n; ++i) {
            double t = 0.0;
            for (int64_t k = 0; k <= i; ++k) t += L[i * n + k] * E[c * n + k];
            out[c * n + i] = mu + t;
        }
    }
    free(E);
}

/*
 * Realisations of the latent process at m new locations conditional on the
 * data (posterior draws): with K the n x m cross covariance, W = L^{-1} K and
 * K** the m x m covariance of the new locations (no nugget),
 *   S  = K** - W^T W           (posterior covariance)
 *   S  = L* L*^T               (unpivoted Cholesky: a pivot <= 0 fails, Sec. 5)
 *   out[c * m + j] = mean_j + (L* e_c)_j,  e_c the normals of realisation
 *   first + c in stream 1, mean as orc_predict.
 * Returns ORC_OK, or ORC_NOT_PD with *info = failing column + 1.
 */
int orc_simulate_conditional(const double *x, int64_t n, const double *xs, int64_t m, int kind,
                             double s2, double rho, const double *L, const double *alpha,
                             double mu_new, int64_t r, uint64_t seed, uint64_t first, double *out,
                             int64_t *info) {
    double *K = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double *W = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);  /* W[j * n + i] */
    double *S = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
    double *mean = (double *)malloc(sizeof(double) * (size_t)m);
    double *E = (double *)malloc(sizeof(double) * (size_t)m * (size_t)r);
    int st = ORC_OK;
    *info = 0;
    orc_cross_cov(x, n, xs, m, kind, s2, rho, K);
    orc_predict(x, n, xs, m, kind, s2, rho, L, alpha, mu_new, mean, NULL);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        double *kc = (double *)malloc(sizeof(double) * (size_t)n);
        for (int64_t i = 0; i < n; ++i) kc[i] = K[i * m + j];
        orc_forward(L, n, kc, W + j * n);
        free(kc);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < m; ++a) {
        for (int64_t b = 0; b < m; ++b) {
            const double kab = (a == b) ? s2 : s2 * orc_kernel(kind, dist2d(xs, a, b) / rho);
            S[a * m + b] = kab - orc_dot(W + a * n, W + b * n, n);
        }
    }
    const int64_t f = orc_cholesky(S, m);
    if (f != 0) {
        *info = f;
        for (int64_t i = 0; i < m * r; ++i) out[i] = NAN;
        st = ORC_NOT_PD;
    } else {
        orc_normals(m, r, seed, 1, first, E);
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < r; ++c) {
            for (int64_t j = 0; j < m; ++j) {
                double t = 0.0;
                for (int64_t k = 0; k <= j; ++k) t += S[j * m + k] * E[c * m + k];
                out[c * m + j] = mean[j] + t;
            }
        }
    }
    free(K); free(W); free(S); free(mean); free(E);
    return st;
}

/*
 * The paper's example covariance (Sec. 4.2): the flux Y_i at phase t_i and
 * log wavelength w_i is a Gaussian-process value plus a random effect of its
 * phase plus measurement error of known variance v_i, so
 *   C_ij = s2 k(|t_i - t_j| / rho_t) k(|w_i - w_j| / rho_w)
 *          + tau2 [t_i == t_j] + v_i [i == j],
 * a separable product of two Matern correlations of smoothness nu = 2, taken
 * here in the Rasmussen & Williams scaling a = sqrt(2 nu) u = 2u:
 *   k(u) = (2^{1-nu} / Gamma(nu)) a^nu K_nu(a) = a^2 K_2(a) / 2,  k(0) = 1.
 * Its derivative in log rho is -u k'(u) = a^3 K_1(a) / 2 (from
 * d/da [a^2 K_2(a)] = -a^2 K_1(a)).
 *
 * K_nu(x), x > 0, from its integral representation
 *   K_nu(x) = int_0^inf exp(-x cosh s) cosh(nu s) ds
 *           = exp(-x) int_0^inf exp(-2 x sinh^2(s/2)) cosh(nu s) ds
 * by the trapezoidal rule with step min(1/16, 1/(4 sqrt(x))) (the integrand
 * is analytic in the strip |Im s| < pi/2 and decays double exponentially, so
 * the rule's error falls like exp(-pi^2 / h); for large x it is a peak of
 * width about 1/sqrt(x), which the step resolves), summed until the terms
 * vanish.
 */
double orc_bessel_k(double nu, double x) {
    if (!(x > 0.0)) return INFINITY;
    /* exp(-x cosh s) = exp(-x) exp(-2 x sinh^2(s/2)): the factor exp(-x) is
       taken out so that large x keeps its relative accuracy */
    /* for large x the integrand is a peak of width about 1/sqrt(x) at s = 0:
       the step shrinks with it (error about exp(-2 pi^2 / (x h^2))) */
    const double h = fmin(1.0 / 16.0, 0.25 / sqrt(x));
    nsum_t s;
    ns_init(&s);
    ns_add(&s, 0.5);
    for (int64_t k = 1; k < 100000; ++k) {
        const double t = h * (double)k;
        const double sh = sinh(0.5 * t);
        const double e = 2.0 * x * sh * sh;
        const double term = exp(-e) * cosh(nu * t);
        ns_add(&s, term);
        if (term < 1e-30 * ns_get(&s) && e > 1.0) break;
    }
    return exp(-x) * h * ns_get(&s);
}

/* k(u) = a^2 K_2(a) / 2, a = 2u (Matern nu = 2) */
double orc_matern2(double u) {
    if (u == 0.0) return 1.0;
    const double a = 2.0 * u;
    return 0.5 * a * a * orc_bessel_k(2.0, a);
}

/* -u k'(u) = a^3 K_1(a) / 2 */
double orc_matern2_dlogrho(double u) {
    if (u == 0.0) return 0.0;
    const double a = 2.0 * u;
    return 0.5 * a * a * a * orc_bessel_k(1.0, a);
}

/* C of the product model, full symmetric n x n (v may be NULL: all zero) */
void orc_prod_cov_fill(const double *x, int64_t n, const double *v, double s2, double rho_t,
                       double rho_w, double tau2, double *C) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            const double dt = fabs(x[2 * i] - x[2 * j]), dw = fabs(x[2 * i + 1] - x[2 * j + 1]);
            double c = s2 * orc_matern2(dt / rho_t) * orc_matern2(dw / rho_w);
            if (dt == 0.0) c += tau2;
            if (i == j && v) c += v[i];
            C[i * n + j] = c;
        }
    }
}

/*
 * Log-likelihood (out[0..2] as orc_loglik) and its gradient with respect to
 * (log s2, log rho_t, log rho_w, log tau2) of the product model:
 *   dC/dlog s2    = s2 k_t k_w
 *   dC/dlog rho_t = s2 (-u_t k'(u_t)) k_w,   dC/dlog rho_w = s2 k_t (-u_w k'(u_w))
 *   dC/dlog tau2  = tau2 [t_i == t_j]
 *   g_j = 1/2 alpha^T dC_j alpha - 1/2 sum_{i,k} W_ik (dC_j)_ik,  W = C^{-1}.
 */
int orc_prod_loglik_grad(const double *x, const double *y, const double *mu, const double *v,
                         int64_t n, double s2, double rho_t, double rho_w, double tau2,
                         double *out, double *alpha, double *grad, int64_t *info) {
    if (info) *info = 0;
    if (n < 1 || !(s2 > 0.0) || !(rho_t > 0.0) || !(rho_w > 0.0) || !(tau2 >= 0.0))
        return ORC_INVALID;
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!isfinite(x[i])) return ORC_INVALID;
    const size_t nn = (size_t)n * (size_t)n;
    double *C = (double *)malloc(sizeof(double) * nn);
    double *L = (double *)malloc(sizeof(double) * nn);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *a = (double *)malloc(sizeof(double) * (size_t)n);
    orc_prod_cov_fill(x, n, v, s2, rho_t, rho_w, tau2, C);
    memcpy(L, C, sizeof(double) * nn);
    const int64_t f = orc_cholesky(L, n);
    if (f != 0) {
        if (info) *info = f;
        out[0] = out[1] = out[2] = NAN;
        if (grad) grad[0] = grad[1] = grad[2] = grad[3] = NAN;
        free(C); free(L); free(r); free(w); free(a);
        return ORC_NOT_PD;
    }
    for (int64_t i = 0; i < n; ++i) r[i] = y[i] - (mu ? mu[i] : 0.0);
    orc_forward(L, n, r, w);
    const double logdet = orc_logdet(L, n), q = orc_dot(w, w, n);
    out[0] = -0.5 * logdet - 0.5 * q - 0.5 * (double)n * log(2.0 * M_PI);
    out[1] = logdet;
    out[2] = q;
    orc_backward(L, n, w, a);
    if (alpha) memcpy(alpha, a, sizeof(double) * (size_t)n);
    if (grad) {
        double *W = (double *)malloc(sizeof(double) * nn);
        orc_inverse_from_chol(L, n, W);
        double *part = (double *)calloc((size_t)n * 4, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            nsum_t g[4];
            for (int c = 0; c < 4; ++c) ns_init(&g[c]);
            for (int64_t j = 0; j < n; ++j) {
                const double dt = fabs(x[2 * i] - x[2 * j]), dw = fabs(x[2 * i + 1] - x[2 * j + 1]);
                const double kt = orc_matern2(dt / rho_t), kw = orc_matern2(dw / rho_w);
                const double d[4] = {s2 * kt * kw, s2 * orc_matern2_dlogrho(dt / rho_t) * kw,
                                     s2 * kt * orc_matern2_dlogrho(dw / rho_w),
                                     dt == 0.0 ? tau2 : 0.0};
                const double cbar = 0.5 * (a[i] * a[j] - W[i * n + j]);
                for (int c = 0; c < 4; ++c) ns_add(&g[c], cbar * d[c]);
            }
            for (int c = 0; c < 4; ++c) part[4 * i + c] = ns_get(&g[c]);
        }
        for (int c = 0; c < 4; ++c) {
            nsum_t s;
            ns_init(&s);
            for (int64_t i = 0; i < n; ++i) ns_add(&s, part[4 * i + c]);
            grad[c] = ns_get(&s);
        }
        free(part);
        free(W);
    }
    free(C); free(L); free(r); free(w); free(a);
    return ORC_OK;
}
