// predict.cu -- kriging prediction at new locations from the factor and alpha
// of a log-likelihood evaluation (Sec. 1: prediction is the conditional
// expectation of the latent process given the data, with its variance;
// Sec. 2.2.2: the cached Cholesky factor is reused through triangular
// solves; Sec. 4.3: predictions with standard errors on a grid).
//
// For new locations xs_1..xs_m, with K_ij = sigma2 k(|x_i - xs_j| / rho)
// (latent process: no nugget between a new and a training location):
//   mean  m_j = mu_new + sum_i K_ij alpha_i                      (matrix-free)
//   var   v_j = sigma2 - |L^{-1} K_.j|^2                          (optional)
//
// The mean never stores K: one thread per new location sweeps the training
// locations and alpha, staged through shared memory in tiles, with the
// table-driven FP64 kernel evaluation of the fill and a compensated sum.
// The variance forms K in chunks of up to PRED_MB new locations (n_p x mb,
// padding rows zero, where L is the identity), solves L V = K by blocks of
// 512 rows, left-looking:
//     V_I = L_II^{-1} (K_I - L_{I,0:I} V_{0:I}),
// with the diagonal-block inverses formed once per call (FP64 blocked
// TRTRI) and both products on the FP64 GEMM, then takes each column's
// squared norm with a compensated warp reduction.  The variance costs
// n_p^2 m flops on the FP64 pipe.
#include <algorithm>

#include "internal.h"
#include "kern.cuh"

namespace gp {

constexpr int PRED_T = 128;      // new locations per CTA of the mean
constexpr int PRED_TILE = 512;   // training locations staged per step
constexpr int64_t PRED_NB = 512; // row blocks of the solve
constexpr int64_t PRED_MB = 2048;  // new locations per variance chunk

struct PSum {
    double s = 0.0, c = 0.0;
    __device__ void add(double x) {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
};

__global__ void __launch_bounds__(PRED_T) predict_mean_kernel(const double2 *__restrict__ x,
                                                              int64_t n,
                                                              const double2 *__restrict__ xs,
                                                              int64_t m, KernParams kp,
                                                              const double *__restrict__ alpha,
                                                              double mu_new, double *mean,
                                                              int64_t *info) {
    __shared__ double tab[EXP_TAB];
    __shared__ double2 xt[PRED_TILE];
    __shared__ double at[PRED_TILE];
    stage_exp_table(kp, tab);
    const int64_t j = (int64_t)blockIdx.x * PRED_T + threadIdx.x;
    double2 p = make_double2(0.0, 0.0);
    if (j < m) {
        p = xs[j];
        if (!isfinite(p.x) || !isfinite(p.y)) set_info(info, -2);
    }
    PSum s;
    for (int64_t i0 = 0; i0 < n; i0 += PRED_TILE) {
        const int cnt = (n - i0) < PRED_TILE ? (int)(n - i0) : PRED_TILE;
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += PRED_T) {
            const double2 t = x[i0 + q];
            if (blockIdx.x == 0 && (!isfinite(t.x) || !isfinite(t.y))) set_info(info, -2);
            xt[q] = t;
            at[q] = alpha[i0 + q];
        }
        __syncthreads();
        for (int q = 0; q < cnt; ++q) s.add(cov_offdiag(kp, pair_dist(xt[q], p), tab) * at[q]);
    }
    if (j < m) mean[j] = mu_new + (s.s + s.c);
}

// After a device-side failure (*info != 0): every output NaN.
__global__ void nan_on_failure_kernel(const int64_t *info, double *a, int64_t na, double *b,
                                      int64_t nb) {
    if (*info == 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < na + nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < na) a[i] = nan("");
        else if (b) b[i - na] = nan("");
    }
}

// B[i + c ldb] = K(i, j0 + c) for i < n, 0 for n <= i < np.
__global__ void __launch_bounds__(256) cross_cov_kernel(const double2 *__restrict__ x, int64_t n,
                                                        int64_t np, const double2 *__restrict__ xs,
                                                        int64_t j0, KernParams kp, double *B,
                                                        int64_t ldb) {
    __shared__ double tab[EXP_TAB];
    stage_exp_table(kp, tab);
    __syncthreads();
    const int64_t c = blockIdx.y;
    const double2 p = xs[j0 + c];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x)
        B[i + c * ldb] = i < n ? cov_offdiag(kp, pair_dist(x[i], p), tab) : 0.0;
}

// var[c] = sigma2 - sum_i V(i, c)^2, one warp per column, compensated.
__global__ void __launch_bounds__(256) column_var_kernel(const double *V, int64_t ldv, int64_t rows,
                                                         int64_t cols, double s2, double *var) {
    const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= cols) return;
    PSum s;
    for (int64_t i = lane; i < rows; i += 32) {
        const double v = V[i + c * ldv];
        s.add(v * v);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s2o = __shfl_xor_sync(0xffffffffu, s.s, off);
        const double c2o = __shfl_xor_sync(0xffffffffu, s.c, off);
        s.add(s2o);
        s.c += c2o;
    }
    if (lane == 0) var[c] = s2 - (s.s + s.c);
}

struct PredWs {
    double *W = nullptr;    // diagonal-block inverses, PRED_NB x PRED_NB each
    double *tmp = nullptr;  // TB x PRED_NB (TRTRI scratch)
    double *B = nullptr;    // n_p x mb: K, then V = L^{-1} K
    double *T = nullptr;    // PRED_NB x mb
    size_t bytes = 0;
};

static PredWs pred_layout(void *base, int64_t np, int64_t mb) {
    PredWs w;
    char *b = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        char *p = b ? b + off : nullptr;
        off += bytes;
        return reinterpret_cast<double *>(p);
    };
    const int64_t nblk = ceil_div(np, PRED_NB);
    w.W = take(sizeof(double) * (size_t)nblk * PRED_NB * PRED_NB);
    w.tmp = take(sizeof(double) * TB * PRED_NB);
    w.B = take(sizeof(double) * (size_t)np * (size_t)mb);
    w.T = take(sizeof(double) * PRED_NB * (size_t)mb);
    w.bytes = (off + 255) & ~size_t(255);
    return w;
}

size_t predict_ws_bytes(int64_t n, int64_t m, int want_var) {
    if (!want_var) return 0;
    return pred_layout(nullptr, round_up(n, PAD), m < PRED_MB ? m : PRED_MB).bytes;
}

static int predict_var(const double2 *x, int64_t n, int64_t np, const double2 *xs, int64_t m,
                       const KernParams &kp, const double *d_L, int64_t ldl, double *d_var,
                       void *d_ws, int64_t *d_info, cudaStream_t s);
int pred_mean_launch(const double2 *x, int64_t n, const double2 *xs, int64_t m, const KernParams &kp,
                     const double *d_alpha, double mu_new, double *d_mean, int64_t *d_info,
                     cudaStream_t s);

int predict_run(const double *d_x, int64_t n, const double *d_xs, int64_t m, const KernParams &kp,
                const double *d_alpha, const double *d_L, int64_t ldl, double mu_new,
                double *d_mean, double *d_var, void *d_ws, int64_t *d_info, cudaStream_t s) {
    const int64_t np = round_up(n, PAD);
    if (cudaMemsetAsync(d_info, 0, sizeof(int64_t), s) != cudaSuccess) return GP_ERR_CUDA;
    const double2 *x = reinterpret_cast<const double2 *>(d_x);
    const double2 *xs = reinterpret_cast<const double2 *>(d_xs);
    GP_TRY(pred_mean_launch(x, n, xs, m, kp, d_alpha, mu_new, d_mean, d_info, s));
    if (d_var) GP_TRY(predict_var(x, n, np, xs, m, kp, d_L, ldl, d_var, d_ws, d_info, s));
    nan_on_failure_kernel<<<(unsigned)std::min<int64_t>(ceil_div(2 * m, 256), 1024), 256, 0, s>>>(
        d_info, d_mean, m, d_var, d_var ? m : 0);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

// W: the inverses of the 512-row diagonal blocks of L (PRED_NB x PRED_NB each).
int pred_block_inverses(const double *d_L, int64_t ldl, int64_t np, double *W, double *tmp,
                        int64_t *d_info, cudaStream_t s) {
    for (int64_t k0 = 0; k0 < np; k0 += PRED_NB) {
        const int64_t nb = (np - k0) < PRED_NB ? (np - k0) : PRED_NB;
        GP_TRY(trtri_fp64_blocked(d_L + k0 + k0 * ldl, ldl, nb, W + (k0 / PRED_NB) * PRED_NB * PRED_NB,
                                  nb, tmp, d_info, s));
    }
    return GP_OK;
}

// B (n_p x mc, ld n_p) = L^{-1} K(:, j0 .. j0 + mc): the cross covariance,
// then the left-looking block solve with the block inverses W; T: PRED_NB x mc.
int pred_solve_cross(const double2 *x, int64_t n, int64_t np, const double2 *xs, int64_t j0,
                     int64_t mc, const KernParams &kp, const double *d_L, int64_t ldl,
                     const double *W, double *B, double *T, int64_t *d_info, cudaStream_t s) {
    dim3 g((unsigned)ceil_div(np, 256 * 4), (unsigned)mc);
    cross_cov_kernel<<<g, 256, 0, s>>>(x, n, np, xs, j0, kp, B, np);
    GP_LAUNCH_CHECK();
    for (int64_t k0 = 0; k0 < np; k0 += PRED_NB) {
        const int64_t nb = (np - k0) < PRED_NB ? (np - k0) : PRED_NB;
        // K_I -= L_{I, 0:I} V_{0:I}
        if (k0 > 0)
            GP_TRY(gemm_f64(nb, mc, k0, -1.0, d_L + k0, ldl, 0, B, np, 0, 1.0, B + k0, np, 0, d_info,
                            s));
        // V_I = L_II^{-1} K_I  (through T)
        const double *Wk = W + (k0 / PRED_NB) * PRED_NB * PRED_NB;
        GP_TRY(gemm_f64(nb, mc, nb, 1.0, Wk, nb, 0, B + k0, np, 0, 0.0, T, nb, 0, d_info, s));
        if (cudaMemcpy2DAsync(B + k0, sizeof(double) * np, T, sizeof(double) * nb,
                              sizeof(double) * nb, mc, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return GP_ERR_CUDA;
    }
    return GP_OK;
}

static int predict_var(const double2 *x, int64_t n, int64_t np, const double2 *xs, int64_t m,
                       const KernParams &kp, const double *d_L, int64_t ldl, double *d_var,
                       void *d_ws, int64_t *d_info, cudaStream_t s) {
    const int64_t mb = m < PRED_MB ? m : PRED_MB;
    PredWs w = pred_layout(d_ws, np, mb);
    GP_TRY(pred_block_inverses(d_L, ldl, np, w.W, w.tmp, d_info, s));
    for (int64_t j0 = 0; j0 < m; j0 += mb) {
        const int64_t mc = (m - j0) < mb ? (m - j0) : mb;
        GP_TRY(pred_solve_cross(x, n, np, xs, j0, mc, kp, d_L, ldl, w.W, w.B, w.T, d_info, s));
        column_var_kernel<<<(unsigned)ceil_div(mc, 8), 256, 0, s>>>(w.B, np, np, mc, kp.s2,
                                                                    d_var + j0);
        GP_LAUNCH_CHECK();
    }
    return GP_OK;
}

int pred_mean_launch(const double2 *x, int64_t n, const double2 *xs, int64_t m, const KernParams &kp,
                     const double *d_alpha, double mu_new, double *d_mean, int64_t *d_info,
                     cudaStream_t s) {
    predict_mean_kernel<<<(unsigned)ceil_div(m, PRED_T), PRED_T, 0, s>>>(x, n, xs, m, kp, d_alpha,
                                                                        mu_new, d_mean, d_info);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

}  // namespace gp
