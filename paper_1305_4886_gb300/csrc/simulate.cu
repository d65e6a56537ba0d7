// simulate.cu -- realisations of the Gaussian process (Sec. 1: unconditional
// realisations and realisations conditional on the data; Sec. 2.3.2: the
// Cholesky factor multiplied by a matrix of standard normals; Sec. 4.3:
// 1000 posterior realisations on the prediction grid).
//
// Standard normals come from the counter-based generator Philox4x64-10
// (Salmon, Moraes, Dror and Shaw, SC 2011), so that every draw is a pure
// function of (seed, stream, realisation, row) and any thread can make any
// draw: for realisation c and rows 4q .. 4q+3 the block function of
// counter (q, c, stream, 0) and key (seed, 0) gives four 64-bit words w_k,
// u_k = ((w_k >> 11) + 1/2) 2^-53, and the Box-Muller transform turns
// (u0, u1) and (u2, u3) into two pairs of normals.  (The paper's package
// uses L'Ecuyer's generator through rlecuyer; the draws are defined by this
// generator instead.)
//
//   unconditional   out_.c = mu + L e_c                       (stream 0)
//   conditional     S = K** - V^T V,  V = L^{-1} K  (posterior covariance of
//                   the latent process at the new locations), S = L* L*^T
//                   (unpivoted FP64 Cholesky: a pivot <= 0 fails, Sec. 5),
//                   out_.c = mean + L* e_c                     (stream 1)
// The products with the triangular factors run on the FP64 GEMM with the
// factor's upper part masked (never read).
#include "internal.h"
#include "kern.cuh"

namespace gp {

struct Philox4 {
    uint64_t w[4];
};

__device__ __forceinline__ Philox4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                 uint64_t k0, uint64_t k1) {
    constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
        c0 = y0;
        c1 = lo1;
        c2 = y2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    Philox4 r;
    r.w[0] = c0;
    r.w[1] = c1;
    r.w[2] = c2;
    r.w[3] = c3;
    return r;
}

__device__ __forceinline__ double u01_open(uint64_t w) {
    return (static_cast<double>(w >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// out[i + c ldo] = z_i of realisation first + c, i < n; rows n .. rows-1 zero.
__global__ void __launch_bounds__(256) rng_normal_kernel(int64_t n, int64_t rows, int64_t r,
                                                         uint64_t seed, uint64_t stream,
                                                         uint64_t first, double *out, int64_t ldo) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (4 * q >= rows) return;
    for (int64_t c = blockIdx.y; c < r; c += gridDim.y) {
        double z[4] = {0.0, 0.0, 0.0, 0.0};
        if (4 * q < n) {
            const Philox4 p = philox4x64_10((uint64_t)q, first + (uint64_t)c, stream, 0, seed, 0);
            const double s0 = sqrt(-2.0 * log(u01_open(p.w[0])));
            const double s2 = sqrt(-2.0 * log(u01_open(p.w[2])));
            double sn, cs;
            sincospi(2.0 * u01_open(p.w[1]), &sn, &cs);
            z[0] = s0 * cs;
            z[1] = s0 * sn;
            sincospi(2.0 * u01_open(p.w[3]), &sn, &cs);
            z[2] = s2 * cs;
            z[3] = s2 * sn;
        }
        double *o = out + c * ldo;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (4 * q + k < rows) o[4 * q + k] = 4 * q + k < n ? z[k] : 0.0;
    }
}

// out[j + c ldo] = (mean ? mean[j] : mu), j < m, c < r.
__global__ void fill_columns_kernel(double *out, int64_t ldo, int64_t m, int64_t r,
                                    const double *mean, double mu) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double v = mean ? mean[j] : mu;
    for (int64_t c = blockIdx.y; c < r; c += gridDim.y) out[j + c * ldo] = v;
}

// NaN into an m x r block when *info != 0.
__global__ void nan_block_kernel(const int64_t *info, double *out, int64_t ldo, int64_t m,
                                 int64_t r) {
    if (*info == 0) return;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (int64_t c = blockIdx.y; c < r; c += gridDim.y) out[j + c * ldo] = nan("");
}

static unsigned grid_y(int64_t r) { return (unsigned)(r < 65535 ? r : 65535); }

int rng_normals(int64_t n, int64_t rows, int64_t r, uint64_t seed, uint64_t stream, uint64_t first,
                double *out, int64_t ldo, cudaStream_t s) {
    dim3 g((unsigned)ceil_div(ceil_div(rows, 4), 256), grid_y(r));
    rng_normal_kernel<<<g, 256, 0, s>>>(n, rows, r, seed, stream, first, out, ldo);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

// out (m x r, ldo) = base + T E with T lower (ldt; upper part never read),
// E (m x r, lde); base: mean[j] (nullable) or mu.
static int lower_times(const double *T, int64_t ldt, int64_t m, const double *E, int64_t lde,
                       int64_t r, const double *mean, double mu, double *out, int64_t ldo,
                       const int64_t *info, cudaStream_t s) {
    fill_columns_kernel<<<dim3((unsigned)ceil_div(m, 256), grid_y(r)), 256, 0, s>>>(out, ldo, m, r,
                                                                                     mean, mu);
    GP_LAUNCH_CHECK();
    F64Mask tri{0, 0, 0, 0, 0};
    tri.a_lower = 1;
    return gemm_f64_ex(m, r, m, 1.0, T, ldt, 0, E, lde, 0, 1.0, out, ldo, 0, tri, info, s);
}

size_t simulate_ws_bytes(int64_t n, int64_t r) {
    return (sizeof(double) * (size_t)n * (size_t)r + 255) & ~size_t(255);
}

int simulate_run(const double *d_L, int64_t n, int64_t ldl, int64_t r, uint64_t seed,
                 uint64_t first, double mu, double *d_out, int64_t ldo, void *d_ws, cudaStream_t s) {
    double *E = static_cast<double *>(d_ws);
    GP_TRY(rng_normals(n, n, r, seed, 0, first, E, n, s));
    return lower_times(d_L, ldl, n, E, n, r, nullptr, mu, d_out, ldo, nullptr, s);
}

// conditional: workspace carving
struct CondWs {
    double *W = nullptr, *tmp = nullptr, *V = nullptr, *T = nullptr, *S = nullptr, *mean = nullptr,
           *E = nullptr;
    size_t bytes = 0;
};

constexpr int64_t SIM_NB = 512;   // row blocks of the solve (as the prediction's)
constexpr int64_t SIM_MB = 2048;  // new locations per solve chunk

static CondWs cond_layout(void *base, int64_t n, int64_t m, int64_t r) {
    CondWs w;
    const int64_t np = round_up(n, PAD), mp = round_up(m, PAD);
    char *b = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t count) {
        off = (off + 255) & ~size_t(255);
        double *p = b ? reinterpret_cast<double *>(b + off) : nullptr;
        off += sizeof(double) * count;
        return p;
    };
    w.W = take((size_t)ceil_div(np, SIM_NB) * SIM_NB * SIM_NB);
    w.tmp = take((size_t)TB * SIM_NB);
    w.V = take((size_t)np * (size_t)m);
    w.T = take((size_t)SIM_NB * (size_t)(m < SIM_MB ? m : SIM_MB));
    w.S = take((size_t)mp * (size_t)mp);
    w.mean = take((size_t)m);
    w.E = take((size_t)m * (size_t)r);
    w.bytes = (off + 255) & ~size_t(255);
    return w;
}

size_t simulate_cond_ws_bytes(int64_t n, int64_t m, int64_t r) {
    return cond_layout(nullptr, n, m, r).bytes;
}

// predict.cu
int pred_block_inverses(const double *d_L, int64_t ldl, int64_t np, double *W, double *tmp,
                        int64_t *d_info, cudaStream_t s);
int pred_solve_cross(const double2 *x, int64_t n, int64_t np, const double2 *xs, int64_t j0,
                     int64_t mc, const KernParams &kp, const double *d_L, int64_t ldl,
                     const double *W, double *B, double *T, int64_t *d_info, cudaStream_t s);
int pred_mean_launch(const double2 *x, int64_t n, const double2 *xs, int64_t m, const KernParams &kp,
                     const double *d_alpha, double mu_new, double *d_mean, int64_t *d_info,
                     cudaStream_t s);

int simulate_cond_run(const double *d_x, int64_t n, const double *d_xs, int64_t m,
                      const gp_params &prm, const double *d_alpha, const double *d_L, int64_t ldl,
                      double mu_new, int64_t r, uint64_t seed, uint64_t first, double *d_out,
                      int64_t ldo, void *d_ws, int64_t *d_info, cudaStream_t s) {
    const int64_t np = round_up(n, PAD), mp = round_up(m, PAD);
    CondWs w = cond_layout(d_ws, n, m, r);
    const double2 *x = reinterpret_cast<const double2 *>(d_x);
    const double2 *xs = reinterpret_cast<const double2 *>(d_xs);
    const KernParams kp = make_kern(prm);
    gp_params latent = prm;
    latent.tau2 = 0.0;  // the new locations' own covariance: latent process, no nugget
    const KernParams kq = make_kern(latent);
    if (cudaMemsetAsync(d_info, 0, sizeof(int64_t), s) != cudaSuccess) return GP_ERR_CUDA;
    GP_TRY(pred_mean_launch(x, n, xs, m, kp, d_alpha, mu_new, w.mean, d_info, s));
    GP_TRY(pred_block_inverses(d_L, ldl, np, w.W, w.tmp, d_info, s));
    for (int64_t j0 = 0; j0 < m; j0 += SIM_MB) {
        const int64_t mc = (m - j0) < SIM_MB ? (m - j0) : SIM_MB;
        GP_TRY(pred_solve_cross(x, n, np, xs, j0, mc, kp, d_L, ldl, w.W, w.V + j0 * np, w.T, d_info,
                                s));
    }
    // S = K** - V^T V (lower), then its factor in place
    GP_TRY(launch_cov_fill(d_xs, m, mp, kq, w.S, mp, d_info, s));
    GP_TRY(gemm_f64(m, m, np, -1.0, w.V, np, 1, w.V, np, 0, 1.0, w.S, mp, 1, d_info, s));
    GP_TRY(chol_fp64_tiled(w.S, mp, mp, 0, d_info, s));
    GP_TRY(rng_normals(m, m, r, seed, 1, first, w.E, m, s));
    GP_TRY(lower_times(w.S, mp, m, w.E, m, r, w.mean, 0.0, d_out, ldo, d_info, s));
    nan_block_kernel<<<dim3((unsigned)ceil_div(m, 256), grid_y(r)), 256, 0, s>>>(d_info, d_out, ldo,
                                                                                  m, r);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

}  // namespace gp
