// solve.cu -- triangular solves with the Cholesky factor, L z products and
// the final reductions (Sec. 1: v = L^{-1}(y - mu); Sec. 2.2.2: the sum of
// squares v^T v and the log-determinant 2 sum log L_ii).
//
// The blocked solves sweep 64-row tiles.  Per tile, one CTA solves the
// 64 x 64 diagonal triangle with a single warp (the solution vector lives in
// registers, two entries per lane, and each solved entry is broadcast with a
// warp shuffle); a second launch applies the tile's GEMV update to every
// remaining row (forward: the column block below the tile, read as
// contiguous column segments; backward: the row block of the tile, one warp
// per column).  Every pass reads L once; the path is HBM-bound.
#include "internal.h"

namespace gp {

// r_i = y_i - mu_i for i < n, 0 for n <= i < np; non-finite data sets info=-2.
__global__ void residual_kernel(const double *y, const double *mu, int64_t n, int64_t np, double *r,
                                int64_t *info) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    double v = 0.0;
    if (i < n) {
        double yi = y[i], mi = mu ? mu[i] : 0.0;
        if (!isfinite(yi) || !isfinite(mi)) set_info(info, -2);
        v = yi - mi;
    }
    r[i] = v;
}

int launch_residual(const double *y, const double *mu, int64_t n, int64_t np, double *r,
                    int64_t *info, cudaStream_t s) {
    residual_kernel<<<(unsigned)ceil_div(np, 256), 256, 0, s>>>(y, mu, n, np, r, info);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

// ---------------------------------------------------------------------------
// Diagonal-tile solves, one warp, lane l owns rows l and l+32.
// trans = 0: b <- L_tt^{-1} b (forward); trans = 1: b <- L_tt^{-T} b.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) trsv_diag_kernel(const double *L, int64_t ld, int64_t j0,
                                                       int bs, int trans, double *b,
                                                       const int64_t *info, const int *skip) {
    if ((info && failed(info)) || (skip && *skip)) return;
    const int l = threadIdx.x;
    const double *T = L + j0 + j0 * ld;
    double v0 = (l < bs) ? b[j0 + l] : 0.0;
    double v1 = (l + 32 < bs) ? b[j0 + l + 32] : 0.0;
    if (trans == 0) {
        for (int c = 0; c < bs; ++c) {
            // x_c = b_c / L_cc, then b_r -= L_rc x_c for r > c
            double mine = (c < 32) ? v0 : v1;
            double bc = __shfl_sync(0xffffffffu, mine, c & 31);
            double xc = bc / T[c + (int64_t)c * ld];
            if (l == (c & 31)) {
                if (c < 32) v0 = xc; else v1 = xc;
            }
            const double *col = T + (int64_t)c * ld;
            if (l > c && l < bs) v0 -= col[l] * xc;
            if (l + 32 > c && l + 32 < bs) v1 -= col[l + 32] * xc;
        }
    } else {
        for (int c = bs - 1; c >= 0; --c) {
            // x_c = b_c / L_cc, then b_r -= L_cr x_c for r < c
            double mine = (c < 32) ? v0 : v1;
            double bc = __shfl_sync(0xffffffffu, mine, c & 31);
            double xc = bc / T[c + (int64_t)c * ld];
            if (l == (c & 31)) {
                if (c < 32) v0 = xc; else v1 = xc;
            }
            if (l < c) v0 -= T[c + (int64_t)l * ld] * xc;
            if (l + 32 < c) v1 -= T[c + (int64_t)(l + 32) * ld] * xc;
        }
    }
    if (l < bs) b[j0 + l] = v0;
    if (l + 32 < bs) b[j0 + l + 32] = v1;
}

// forward update: b_i -= sum_{c < bs} L[i, j0 + c] x_c for j0+bs <= i < n
__global__ void __launch_bounds__(256) trsv_fwd_update_kernel(const double *L, int64_t ld,
                                                              int64_t j0, int bs, int64_t n,
                                                              double *b, const int64_t *info,
                                                              const int *skip) {
    __shared__ double xs[TB];
    if ((info && failed(info)) || (skip && *skip)) return;
    if (threadIdx.x < bs) xs[threadIdx.x] = b[j0 + threadIdx.x];
    __syncthreads();
    int64_t i = j0 + bs + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *p = L + i + j0 * ld;
    double acc = 0.0;
    for (int c = 0; c < bs; ++c) acc = fma(p[(int64_t)c * ld], xs[c], acc);
    b[i] -= acc;
}

// backward update: b_c -= sum_{r < bs} L[j0 + r, c] x_r for 0 <= c < j0
__global__ void __launch_bounds__(256) trsv_bwd_update_kernel(const double *L, int64_t ld,
                                                              int64_t j0, int bs, double *b,
                                                              const int64_t *info,
                                                              const int *skip) {
    if ((info && failed(info)) || (skip && *skip)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double x0 = (lane < bs) ? b[j0 + lane] : 0.0;
    double x1 = (lane + 32 < bs) ? b[j0 + lane + 32] : 0.0;
    const int64_t cbeg = blockIdx.x * (int64_t)64;
    for (int q = warp; q < 64; q += 8) {
        int64_t c = cbeg + q;
        if (c >= j0) break;
        const double *col = L + j0 + c * ld;
        double acc = 0.0;
        if (lane < bs) acc = col[lane] * x0;
        if (lane + 32 < bs) acc = fma(col[lane + 32], x1, acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) b[c] -= acc;
    }
}

// In-place solve on b (n values): trans = 0 -> L^{-1} b, trans = 1 -> L^{-T} b.
// skip (nullable): a device flag that turns every launch into a no-op.
int trsv_blocked_skip(const double *L, int64_t ld, int64_t n, int trans, double *b,
                      const int64_t *info, const int *skip, cudaStream_t s) {
    const int64_t T = ceil_div(n, TB);
    if (trans == 0) {
        for (int64_t t = 0; t < T; ++t) {
            const int64_t j0 = t * TB;
            const int bs = (int)((n - j0) < TB ? (n - j0) : TB);
            trsv_diag_kernel<<<1, 32, 0, s>>>(L, ld, j0, bs, 0, b, info, skip);
            GP_LAUNCH_CHECK();
            const int64_t rest = n - j0 - bs;
            if (rest > 0) {
                trsv_fwd_update_kernel<<<(unsigned)ceil_div(rest, 256), 256, 0, s>>>(L, ld, j0, bs, n,
                                                                                      b, info, skip);
                GP_LAUNCH_CHECK();
            }
        }
    } else {
        for (int64_t t = T - 1; t >= 0; --t) {
            const int64_t j0 = t * TB;
            const int bs = (int)((n - j0) < TB ? (n - j0) : TB);
            trsv_diag_kernel<<<1, 32, 0, s>>>(L, ld, j0, bs, 1, b, info, skip);
            GP_LAUNCH_CHECK();
            if (j0 > 0) {
                trsv_bwd_update_kernel<<<(unsigned)ceil_div(j0, 64), 256, 0, s>>>(L, ld, j0, bs, b,
                                                                                   info, skip);
                GP_LAUNCH_CHECK();
            }
        }
    }
    return GP_OK;
}

int trsv_blocked(const double *L, int64_t ld, int64_t n, int trans, double *b,
                 const int64_t *info, cudaStream_t s) {
    return trsv_blocked_skip(L, ld, n, trans, b, info, nullptr, s);
}

// ---------------------------------------------------------------------------
// y = L z.  Grid (row blocks of 256, column chunks of 2048); each thread owns
// one row and accumulates its chunk, then adds it atomically (y zeroed
// first).
// ---------------------------------------------------------------------------
constexpr int MV_CHUNK = 2048;

__global__ void __launch_bounds__(256) lower_matvec_kernel(const double *L, int64_t ld, int64_t n,
                                                           const double *z, double *y) {
    __shared__ double zs[MV_CHUNK];
    const int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x;
    const int64_t k0 = blockIdx.y * (int64_t)MV_CHUNK;
    const int64_t rmax = (blockIdx.x + 1) * (int64_t)256 - 1;
    if (k0 > rmax || k0 >= n) return;  // chunk entirely above this row block
    const int64_t k1 = min(min(k0 + MV_CHUNK, n), rmax + 1);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += 256) zs[k - k0] = z[k];
    __syncthreads();
    if (i >= n) return;
    const int64_t kend = min(k1, i + 1);
    double acc = 0.0;
    for (int64_t k = k0; k < kend; ++k) acc = fma(L[i + k * ld], zs[k - k0], acc);
    atomicAdd(y + i, acc);
}

int lower_matvec(const double *L, int64_t ld, int64_t n, const double *z, double *y,
                 cudaStream_t s) {
    if (cudaMemsetAsync(y, 0, sizeof(double) * n, s) != cudaSuccess) return GP_ERR_CUDA;
    dim3 g((unsigned)ceil_div(n, 256), (unsigned)ceil_div(n, MV_CHUNK));
    lower_matvec_kernel<<<g, 256, 0, s>>>(L, ld, n, z, y);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

// ---------------------------------------------------------------------------
// logdet = 2 sum log L_ii and q = u^T v over i < n (Sec. 2.2.2).  Each thread
// keeps Neumaier-compensated sums; the 1024 partial sums are combined by a
// butterfly of warp shuffles (sum and compensation both), then one warp
// combines the 32 warp sums the same way: a fixed order, so the result is
// deterministic.  out = {loglik, logdet, q, resid}; NaN when *info != 0.
// ---------------------------------------------------------------------------
struct NSum {
    double s = 0.0, c = 0.0;
    __device__ void add(double x) {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    // adds another compensated sum (its sum with compensation, its compensation plainly)
    __device__ void merge(double s2, double c2) {
        add(s2);
        c += c2;
    }
    __device__ double get() const { return s + c; }
};

__device__ __forceinline__ void warp_merge(NSum &x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, x.s, off);
        const double c2 = __shfl_xor_sync(0xffffffffu, x.c, off);
        x.merge(s2, c2);
    }
}

__global__ void __launch_bounds__(1024) loglik_reduce_kernel(const double *L, int64_t ld, int64_t n,
                                                             const double *u, const double *v,
                                                             const double *resid, double *out,
                                                             const int64_t *info) {
    __shared__ double ws[4][32];
    NSum a, b;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        a.add(log(L[i + i * ld]));
        b.add(u[i] * v[i]);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    warp_merge(a);
    warp_merge(b);
    if (lane == 0) {
        ws[0][warp] = a.s;
        ws[1][warp] = a.c;
        ws[2][warp] = b.s;
        ws[3][warp] = b.c;
    }
    __syncthreads();
    if (warp != 0) return;
    NSum A, B;
    A.s = ws[0][lane];
    A.c = ws[1][lane];
    B.s = ws[2][lane];
    B.c = ws[3][lane];
    warp_merge(A);
    warp_merge(B);
    if (lane == 0) {
        double logdet = 2.0 * A.get(), q = B.get();
        if (*info != 0) {
            out[0] = out[1] = out[2] = out[3] = nan("");
        } else {
            const double LOG_2PI = 1.8378770664093454836;
            out[0] = -0.5 * logdet - 0.5 * q - 0.5 * (double)n * LOG_2PI;
            out[1] = logdet;
            out[2] = q;
            out[3] = resid ? *resid : 0.0;
        }
    }
}

int launch_loglik_reduce(const double *L, int64_t ld, int64_t n, const double *u, const double *v,
                         const double *resid, double *out, const int64_t *info, cudaStream_t s) {
    loglik_reduce_kernel<<<1, 1024, 0, s>>>(L, ld, n, u, v, resid, out, info);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

}  // namespace gp
