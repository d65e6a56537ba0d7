// refine.cu -- iterative refinement of alpha = C^{-1} r for the mixed form,
// against a matrix-free FP64 residual s = r - C(theta) alpha.
//
// C(theta) is never re-read from memory: every 64 x 64 lower tile is
// recomputed from the locations (the same covariance routine as the fill),
// and applied twice, C_IJ alpha_J to rows I and C_IJ^T alpha_I to rows J,
// so each pair costs one kernel evaluation.  Row and column partial sums are
// reduced in registers/warp shuffles and added to the accumulator with FP64
// atomics.
//
// Refinement (not in the paper): with the mixed factor L~,
//   repeat: s = r - C alpha; stop if ||s|| <= tol ||r||; alpha += L~^{-T} L~^{-1} s
// A device flag records convergence so that later launches of a fixed-length
// sequence return at once (no host round trip).
#include "internal.h"
#include "kern.cuh"

namespace gp {

__global__ void __launch_bounds__(256) cov_matvec_kernel(const double2 *__restrict__ x, int64_t n,
                                                         KernParams kp,
                                                         const double *__restrict__ a, double *acc,
                                                         const int *skip, const int64_t *info) {
    __shared__ double2 xc[TB];
    __shared__ double tab[EXP_TAB];
    stage_exp_table(kp, tab);
    __shared__ double ac[TB];
    __shared__ double colsum[2][TB];
    __shared__ double rowsum[4][TB];
    if ((skip && *skip) || failed(info)) return;
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    if (row0 >= n) return;
    const int tid = threadIdx.x;
    if (tid < TB) {
        int64_t j = col0 + tid;
        xc[tid] = (j < n) ? x[j] : make_double2(0.0, 0.0);
        ac[tid] = (j < n) ? a[j] : 0.0;
        colsum[0][tid] = 0.0;
        colsum[1][tid] = 0.0;
    }
    __syncthreads();
    const int r = tid & (TB - 1);
    const int cg = tid >> 6;
    const int half = (tid >> 5) & 1;
    const int64_t i = row0 + r;
    const bool diag = (ti == tj);
    const bool row_ok = i < n;
    const double2 xi = row_ok ? x[i] : make_double2(0.0, 0.0);
    const double ai = row_ok ? a[i] : 0.0;
    double rs = 0.0;
    for (int c = cg; c < TB; c += 4) {
        const int64_t j = col0 + c;
        double v = 0.0;
        if (row_ok && j < n) v = (i == j) ? kp.diag : cov_offdiag(kp, pair_dist(xi, xc[c]), tab);
        rs = fma(v, ac[c], rs);
        if (!diag) {
            double cs = v * ai;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
            if ((tid & 31) == 0) colsum[half][c] += cs;  // one lane per (warp, column)
        }
    }
    rowsum[cg][r] = rs;
    __syncthreads();
    if (tid < TB) {
        const int64_t ii = row0 + tid;
        if (ii < n) atomicAdd(acc + ii, rowsum[0][tid] + rowsum[1][tid] + rowsum[2][tid] + rowsum[3][tid]);
        if (!diag) {
            const int64_t jj = col0 + tid;
            if (jj < n) atomicAdd(acc + jj, colsum[0][tid] + colsum[1][tid]);
        }
    }
}

// The same symmetric tile matvec with the entries and products in
// double-float on the FP32 pipe (tensor-core forms): row sums per thread,
// column sums by warp shuffles of (hi, lo) pairs, one FP64 atomic per row
// and column of the tile.
__device__ __forceinline__ dfl df_shfl_xor(dfl v, int o) {
    return {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}

__global__ void __launch_bounds__(256) cov_matvec_df_kernel(const double2 *__restrict__ x,
                                                            int64_t n, KernParams kp,
                                                            const double *__restrict__ a,
                                                            double *acc, const int *skip,
                                                            const int64_t *info) {
    __shared__ float4 xc[TB];
    __shared__ float2 tab[DF_TAB];
    __shared__ float2 ac[TB];
    __shared__ float2 colsum[2][TB];
    __shared__ float2 rowsum[4][TB];
    stage_df_table(kp.kd, tab);
    if ((skip && *skip) || failed(info)) return;
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    if (row0 >= n) return;
    const int tid = threadIdx.x;
    if (tid < TB) {
        const int64_t j = col0 + tid;
        xc[tid] = df_point(j < n ? x[j] : make_double2(0.0, 0.0));
        const dfl aj = f64_to_df(static_cast<unsigned long long>(
            __double_as_longlong(j < n ? a[j] : 0.0)));
        ac[tid] = make_float2(aj.h, aj.l);
        colsum[0][tid] = colsum[1][tid] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const int r = tid & (TB - 1);
    const int cg = tid >> 6;
    const int half = (tid >> 5) & 1;
    const int64_t i = row0 + r;
    const bool diag = (ti == tj);
    const bool row_ok = i < n;
    const float4 xi = df_point(row_ok ? x[i] : make_double2(0.0, 0.0));
    const dfl ai = f64_to_df(static_cast<unsigned long long>(__double_as_longlong(row_ok ? a[i] : 0.0)));
    dfl rs{0.0f, 0.0f};
    for (int c = cg; c < TB; c += 4) {
        const int64_t j = col0 + c;
        dfl v{0.0f, 0.0f};
        if (row_ok && j < n) {
            if (i == j) {
                v = kp.kd.diag;
            } else {
                dfl unused;
                df_cov<false>(kp.kind, kp.kd, df_dist(xi, xc[c]), tab, v, unused);
            }
        }
        rs = df_add(rs, df_mul(v, dfl{ac[c].x, ac[c].y}));
        if (!diag) {
            dfl cs = df_mul(v, ai);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cs = df_add(cs, df_shfl_xor(cs, o));
            if ((tid & 31) == 0) colsum[half][c] = make_float2(cs.h, cs.l);  // one warp per (half, c)
        }
    }
    rowsum[cg][r] = make_float2(rs.h, rs.l);
    __syncthreads();
    if (tid < TB) {
        const int64_t ii = row0 + tid;
        if (ii < n) {
            dfl t{rowsum[0][tid].x, rowsum[0][tid].y};
            for (int q = 1; q < 4; ++q) t = df_add(t, dfl{rowsum[q][tid].x, rowsum[q][tid].y});
            atomicAdd(acc + ii, df_to_double(t));
        }
        if (!diag) {
            const int64_t jj = col0 + tid;
            if (jj < n) {
                const dfl t = df_add(dfl{colsum[0][tid].x, colsum[0][tid].y},
                                     dfl{colsum[1][tid].x, colsum[1][tid].y});
                atomicAdd(acc + jj, df_to_double(t));
            }
        }
    }
}

// s = r - acc over i < n; ||s||, ||r|| reduced in one CTA (deterministic);
// stats[0] = ||s|| / ||r||.  Sets *conv when the ratio is <= tol (or r = 0).
__global__ void __launch_bounds__(1024) refine_resid_kernel(const double *r, const double *acc,
                                                            int64_t n, double *s, double tol,
                                                            double *stats, int *conv,
                                                            const int64_t *info) {
    __shared__ double ps[2][1024];
    if (*conv || failed(info)) return;
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        double si = r[i] - acc[i];
        s[i] = si;
        a = fma(si, si, a);
        b = fma(r[i], r[i], b);
    }
    ps[0][threadIdx.x] = a;
    ps[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ps[0][threadIdx.x] += ps[0][threadIdx.x + w];
            ps[1][threadIdx.x] += ps[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double ratio = ps[1][0] > 0.0 ? sqrt(ps[0][0] / ps[1][0]) : 0.0;
        stats[0] = ratio;
        if (ratio <= tol) *conv = 1;
    }
}

__global__ void axpy_kernel(int64_t n, const double *d, double *a, const int *skip,
                            const int64_t *info) {
    if (*skip || failed(info)) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] += d[i];
}

int cov_matvec(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *a,
               double *acc, const int *skip, const int64_t *info, cudaStream_t s) {
    if (cudaMemsetAsync(acc, 0, sizeof(double) * n, s) != cudaSuccess) return GP_ERR_CUDA;
    const int64_t T = np / TB;
    const int ev = prof_start(s);
    if (kp.product)
        GP_TRY(prod_matvec(d_x, n, np, kp, a, acc, skip, info, s));
    else if (kp.use_df)
        cov_matvec_df_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(
            reinterpret_cast<const double2 *>(d_x), n, kp, a, acc, skip, info);
    else
        cov_matvec_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(
            reinterpret_cast<const double2 *>(d_x), n, kp, a, acc, skip, info);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_RESIDUAL, 0.0, 0.0);
    return GP_OK;
}

int refine_alpha(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *L,
                 int64_t ld, const double *r, double *alpha, double *acc, double *s,
                 double *stats, int *conv, int *tsync, int max_evals, double tol, int64_t *info,
                 cudaStream_t st) {
    if (cudaMemsetAsync(conv, 0, sizeof(int), st) != cudaSuccess) return GP_ERR_CUDA;
    for (int it = 0; it < max_evals; ++it) {
        GP_TRY(cov_matvec(d_x, n, np, kp, alpha, acc, conv, info, st));
        refine_resid_kernel<<<1, 1024, 0, st>>>(r, acc, n, s, tol, stats, conv, info);
        GP_LAUNCH_CHECK();
        if (it + 1 == max_evals) break;  // the last evaluation only reports
        GP_TRY(trsv_persist(L, ld, n, 0, s, tsync, info, conv, st));
        GP_TRY(trsv_persist(L, ld, n, 1, s, tsync, info, conv, st));
        axpy_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, s, alpha, conv, info);
        GP_LAUNCH_CHECK();
    }
    return GP_OK;
}

}  // namespace gp
