// fill.cu -- covariance-tile fill (Sec. 1: C = C_g + C_y built from the
// locations; Sec. 2.3.5: entries computed at given indices and stored
// column-wise).
//
// One CTA fills one 64 x 64 lower tile of the column-major n_p x n_p matrix.
// The 64 column locations are staged in shared memory as double2 loads; each
// thread owns one row point in registers and sweeps 16 columns, so a warp
// writes 32 consecutive doubles of one column per store (coalesced).  Only
// tiles with ti >= tj are launched; diagonal tiles are written whole
// (symmetric values), padding rows/columns hold the identity.
#include "internal.h"
#include "kern.cuh"

namespace gp {

__global__ void __launch_bounds__(256) cov_fill_kernel(const double2 *__restrict__ x, int64_t n,
                                                       int64_t tiles_per_side, KernParams kp,
                                                       double *__restrict__ C, int64_t ldc,
                                                       int64_t *info) {
    __shared__ double2 xc[TB];
    __shared__ double tab[EXP_TAB];
    stage_exp_table(kp, tab);
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    (void)tiles_per_side;
    const int64_t row0 = ti * TB, col0 = tj * TB;
    const int tid = threadIdx.x;
    if (tid < TB) {
        int64_t j = col0 + tid;
        double2 p = make_double2(0.0, 0.0);
        if (j < n) {
            p = x[j];
            if (info && (!isfinite(p.x) || !isfinite(p.y))) set_info(info, -2);
        }
        xc[tid] = p;
    }
    __syncthreads();
    const int r = tid & (TB - 1);
    const int cg = tid >> 6;  // 0..3
    const int64_t i = row0 + r;
    double2 xi = make_double2(0.0, 0.0);
    if (i < n) xi = x[i];
    double *col = C + i;
#pragma unroll 4
    for (int c = cg; c < TB; c += 4) {
        const int64_t j = col0 + c;
        double v;
        if (i < n && j < n) {
            v = (i == j) ? kp.diag : cov_offdiag(kp, pair_dist(xi, xc[c]), tab);
        } else {
            v = (i == j) ? 1.0 : 0.0;
        }
        col[j * ldc] = v;
    }
}

// The same tile fill with the off-diagonal entries evaluated in double-float
// on the FP32 pipe (tensor-core forms); one FP64 add per entry assembles the
// value.
__global__ void __launch_bounds__(256) cov_fill_df_kernel(const double2 *__restrict__ x, int64_t n,
                                                          KernParams kp, double *__restrict__ C,
                                                          int64_t ldc, int64_t *info) {
    __shared__ float4 xc[TB];
    __shared__ float2 tab[DF_TAB];
    stage_df_table(kp.kd, tab);
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    const int tid = threadIdx.x;
    if (tid < TB) {
        const int64_t j = col0 + tid;
        double2 p = make_double2(0.0, 0.0);
        if (j < n) {
            p = x[j];
            if (info && (!isfinite(p.x) || !isfinite(p.y))) set_info(info, -2);
        }
        xc[tid] = df_point(p);
    }
    __syncthreads();
    const int r = tid & (TB - 1);
    const int cg = tid >> 6;  // 0..3
    const int64_t i = row0 + r;
    const float4 xi = df_point(i < n ? x[i] : make_double2(0.0, 0.0));
    double *col = C + i;
#pragma unroll 2
    for (int c = cg; c < TB; c += 4) {
        const int64_t j = col0 + c;
        double v;
        if (i < n && j < n) {
            if (i == j) {
                v = kp.diag;
            } else {
                dfl cv, unused;
                df_cov<false>(kp.kind, kp.kd, df_dist(xi, xc[c]), tab, cv, unused);
                v = df_to_double(cv);
            }
        } else {
            v = (i == j) ? 1.0 : 0.0;
        }
        col[j * ldc] = v;
    }
}

int launch_cov_fill(const double *d_x, int64_t n, int64_t np, const KernParams &kp, double *d_C,
                    int64_t ldc, int64_t *d_info, cudaStream_t s) {
    if (kp.product) return prod_fill(d_x, n, np, kp, d_C, ldc, d_info, s);
    const int64_t T = np / TB;
    const int64_t ntiles = T * (T + 1) / 2;
    if (ntiles > 0x7fffffffLL) return GP_ERR_INVALID;
    const int ev = prof_start(s);
    if (kp.use_df)
        cov_fill_df_kernel<<<(unsigned)ntiles, 256, 0, s>>>(reinterpret_cast<const double2 *>(d_x), n,
                                                            kp, d_C, ldc, d_info);
    else
        cov_fill_kernel<<<(unsigned)ntiles, 256, 0, s>>>(reinterpret_cast<const double2 *>(d_x), n,
                                                         T, kp, d_C, ldc, d_info);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_FILL, 0.0, 8.0 * (double)np * (double)(np + 1) / 2.0);
    return GP_OK;
}

}  // namespace gp
