// dense_f64.cu -- FP64 CUDA-core building blocks of the tiled Cholesky
// (Sec. 2.1: factor the diagonal block, forward-solve the blocks below it,
// update the trailing blocks by multiply-and-subtract; repeat per block
// column).
//
//   potrf_tile   Cholesky of one 64 x 64 diagonal tile in shared memory.
//   trsm_tiles   panel solve  B <- B L_kk^{-T}  for the tiles below it.
//   trtri_tiles  inverse of each 64 x 64 diagonal tile of a lower block.
//   gemm_f64     C = alpha op(A) op(B) + beta C, 64 x 64 register-tiled.
//
// GB300 executes FP64 at a small fraction of its tensor rate, so these
// kernels are bounded by the FP64 pipe, not by memory: a 4 x 4 register tile
// per thread keeps shared-memory traffic far below the DFMA issue rate.
#include "internal.h"

namespace gp {

// ---------------------------------------------------------------------------
// Cholesky of the 64 x 64 tile at A (column-major, ld), right-looking in
// shared memory on the unscaled columns: step j subtracts a_rj a_cj / d_j
// from the trailing lower triangle (d_j the current pivot), and the columns
// are scaled by 1/sqrt(d_j) once at the end (L_rj = a_rj / sqrt(d_j)).  Each
// step costs one reciprocal, two barriers and one FMA per trailing lower
// entry (a warp per column: the FP64 pipe of one SM, about two FMAs per
// clock, is what bounds this kernel).  col_base is the global column of the
// tile's first column (for the d_info convention).  A pivot <= 0 or NaN
// stops the factorisation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) potrf_tile_kernel(double *A, int64_t ld, int64_t col_base,
                                                         int64_t *info) {
    __shared__ double S[TB * (TB + 1)];
    __shared__ double lj[TB];    // a_cj / d_j of the current step
    __shared__ double dinv[TB];
    __shared__ int bad;
    if (failed(info)) return;
    const int tid = threadIdx.x;
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        S[c * (TB + 1) + r] = (r >= c) ? A[r + (int64_t)c * ld] : 0.0;
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < TB; ++j) {
        const double *cj = S + j * (TB + 1);
        if (tid < TB) {
            // every thread of the first two warps forms 1/d_j (one division's
            // latency on the serial chain) and its own multiplier
            const double d = cj[j];
            if (!(d > 0.0)) {
                if (tid == 0) {
                    bad = 1;
                    set_info(info, col_base + j + 1);
                }
            } else {
                const double inv = 1.0 / d;
                if (tid == 0) dinv[j] = inv;
                if (tid > j) lj[tid] = cj[tid] * inv;
            }
        }
        __syncthreads();
        if (bad) break;  // uniform
        // a_rc -= a_rj a_cj / d_j on the trailing lower triangle j < c <= r,
        // flattened over all threads (every lane busy: on this FP64 pipe a
        // warp instruction costs the same with few lanes active), one FMA per
        // entry
        const int ntri = (TB - 1 - j) * (TB - j) / 2;
        for (int e = tid; e < ntri; e += blockDim.x) {
            int r, c;
            tri_desc_entry(e, TB, r, c);
            S[c * (TB + 1) + r] = fma(-cj[r], lj[c], S[c * (TB + 1) + r]);
        }
        __syncthreads();
    }
    if (bad) return;
    // L_rj = a_rj / sqrt(d_j):  a_rj * sqrt(1/d_j), one square root per column
    if (tid < TB) dinv[tid] = sqrt(dinv[tid]);
    __syncthreads();
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        if (r >= c) A[r + (int64_t)c * ld] = S[c * (TB + 1) + r] * dinv[c];
    }
}

// ---------------------------------------------------------------------------
// B <- B L^{-T} for the rows below the diagonal tile L (the panel
// forward-solve of Sec. 2.1).  Each CTA solves 32 rows (rows r0 = 32 blockIdx
// of B0) against the whole 64 x 64 triangle; the pivots' reciprocals are
// formed once.
// ---------------------------------------------------------------------------
constexpr int TR_ROWS = 32;

__global__ void __launch_bounds__(256) trsm_tiles_kernel(const double *L, double *B0, int64_t ld,
                                                         int64_t rows, const int64_t *info) {
    __shared__ double Ls[TB * (TB + 1)];
    __shared__ double Bs[TB * (TR_ROWS + 1)];
    __shared__ double rinv[TB];
    if (failed(info)) return;
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * TR_ROWS;
    double *B = B0 + r0;
    const int nr = (int)((rows - r0) < TR_ROWS ? (rows - r0) : TR_ROWS);
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        Ls[c * (TB + 1) + r] = (r >= c) ? L[r + (int64_t)c * ld] : 0.0;
    }
    for (int e = tid; e < TB * TR_ROWS; e += blockDim.x) {
        int r = e & (TR_ROWS - 1), c = e >> 5;
        Bs[c * (TR_ROWS + 1) + r] = (r < nr) ? B[r + (int64_t)c * ld] : 0.0;
    }
    __syncthreads();
    if (tid < TB) rinv[tid] = 1.0 / Ls[tid * (TB + 1) + tid];
    __syncthreads();
    // M_{c2,c} = L_{c2,c} / L_cc, so that on the unscaled columns
    // b_c2 -= b_c M_{c2,c} (X_c = b_c / L_cc is applied once at the end)
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        if (r > c) Ls[c * (TB + 1) + r] *= rinv[c];
    }
    __syncthreads();
    // X L^T = B: column c of X = (B_c - sum_{l<c} X_l L_cl) / L_cc
    for (int c = 0; c < TB - 1; ++c) {
        const int w = TB - 1 - c;
        for (int e = tid; e < w * TR_ROWS; e += blockDim.x) {
            int c2 = c + 1 + e / TR_ROWS;
            int r = e & (TR_ROWS - 1);
            Bs[c2 * (TR_ROWS + 1) + r] -= Bs[c * (TR_ROWS + 1) + r] * Ls[c * (TB + 1) + c2];
        }
        __syncthreads();
    }
    for (int e = tid; e < TB * TR_ROWS; e += blockDim.x) {
        int r = e & (TR_ROWS - 1), c = e >> 5;
        if (r < nr) B[r + (int64_t)c * ld] = Bs[c * (TR_ROWS + 1) + r] * rinv[c];
    }
}

// ---------------------------------------------------------------------------
// X_tt = L_tt^{-1} for every 64 x 64 diagonal tile t of the lower block L
// (ld_l); X (ld_x) receives full tiles with zeros above the diagonal.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) trtri_tiles_kernel(const double *L, int64_t ld_l, double *X,
                                                          int64_t ld_x, const int64_t *info) {
    __shared__ double Ls[TB * (TB + 1)];
    __shared__ double Bs[TB * (TB + 1)];
    if (failed(info)) return;
    const int tid = threadIdx.x;
    const int64_t off = (int64_t)blockIdx.x * TB;
    const double *Lt = L + off + off * ld_l;
    double *Xt = X + off + off * ld_x;
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        Ls[c * (TB + 1) + r] = (r >= c) ? Lt[r + (int64_t)c * ld_l] : 0.0;
        Bs[c * (TB + 1) + r] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    __shared__ double rinv[TB];
    if (tid < TB) rinv[tid] = 1.0 / Ls[tid * (TB + 1) + tid];
    __syncthreads();
    // row c of L scaled by 1/L_cc: on the unscaled columns b_c2 -= b_c L_c,c2 / L_cc,
    // and X_c = b_c / L_cc is applied once at the end
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        if (r > c) Ls[c * (TB + 1) + r] *= rinv[r];
    }
    __syncthreads();
    // X L = I: column c of X (descending) = (B_c - sum_{l>c} X_l L_lc) / L_cc
    for (int c = TB - 1; c > 0; --c) {
        // column c of B is zero above row c: rows c.. only (exact zeros skipped)
        const int nr = TB - c;
        for (int e = tid; e < c * nr; e += blockDim.x) {
            const int c2 = e / nr;
            const int r = c + (e - c2 * nr);
            Bs[c2 * (TB + 1) + r] -= Bs[c * (TB + 1) + r] * Ls[c2 * (TB + 1) + c];
        }
        __syncthreads();
    }
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        Xt[r + (int64_t)c * ld_x] = (r >= c) ? Bs[c * (TB + 1) + r] * rinv[c] : 0.0;
    }
}

// ---------------------------------------------------------------------------
// C (M x N) = alpha op(A) op(B) + beta C, column-major.
//   opA = 0: op(A)(r,k) = A[r + k lda]    opA = 1: A[k + r lda]
//   opB = 0: op(B)(k,c) = B[k + c ldb]    opB = 1: B[c + k ldb]
// lower != 0: M == N and only 64 x 64 tiles with tile row >= tile column are
// computed (grid is the triangular tile count).
// mask.out_lower: write only entries with row + diag_off >= col.
// mask.tri_k: op(B)(k, c) vanishes for k < c - tri_off; tiles start their K
// loop there.
// ---------------------------------------------------------------------------
constexpr int GBK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                       const double *__restrict__ A, int64_t lda,
                                                       int opA, const double *__restrict__ B,
                                                       int64_t ldb, int opB, double beta,
                                                       double *C, int64_t ldc, int lower,
                                                       F64Mask mask, const int64_t *info) {
    __shared__ double As[GBK][TB + 1];
    __shared__ double Bs[GBK][TB + 1];
    if (info && failed(info)) return;
    int64_t bi, bj;
    if (lower) {
        lower_tile_coords(blockIdx.x, bi, bj);
    } else {
        bi = blockIdx.x;
        bj = blockIdx.y;
    }
    const int64_t r0 = bi * TB, c0 = bj * TB;
    if (mask.out_lower && c0 > r0 + (TB - 1) + mask.diag_off) return;
    int64_t kbeg = 0;
    if (mask.tri_k && c0 - mask.tri_off > 0) kbeg = ((c0 - mask.tri_off) / GBK) * GBK;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    for (int64_t k0 = kbeg; k0 < K; k0 += GBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int idx = tid + 256 * q;
            int r, k;
            double v = 0.0;
            if (opA == 0) {
                r = idx & 63;
                k = idx >> 6;
                int64_t gr = r0 + r, gk = k0 + k;
                if (gr < M && gk < K) v = A[gr + gk * lda];
            } else {
                k = idx & 15;
                r = idx >> 4;
                int64_t gr = r0 + r, gk = k0 + k;
                if (gr < M && gk < K) v = A[gk + gr * lda];
            }
            As[k][r] = v;
            double w = 0.0;
            int c, kb;
            if (opB == 0) {
                kb = idx & 15;
                c = idx >> 4;
                int64_t gc = c0 + c, gk = k0 + kb;
                if (gc < N && gk < K) w = B[gk + gc * ldb];
            } else {
                c = idx & 63;
                kb = idx >> 6;
                int64_t gc = c0 + c, gk = k0 + kb;
                if (gc < N && gk < K) w = B[gc + gk * ldb];
            }
            Bs[kb][c] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GBK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[k][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[k][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int64_t gc = c0 + ty + 16 * b;
        if (gc >= N) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int64_t gr = r0 + tx + 16 * a;
            if (gr >= M) continue;
            if (mask.out_lower && gr + mask.diag_off < gc) continue;
            double *p = C + gr + gc * ldc;
            double v = alpha * acc[a][b];
            if (beta != 0.0) v = fma(beta, *p, v);
            *p = v;
        }
    }
}

// 32 x 32 output tiles, 128 threads (2 x 4 per thread): four times the
// CTAs of the 64 x 64 kernel for the small, latency-bound updates of the
// diagonal blocks, and four warps per CTA so that one CTA keeps all four FP64
// sub-pipes of its SM busy.  mask.kchunk > 0 splits K into chunks over
// grid.z and adds each partial product with FP64 atomics (C must already
// hold beta C).
constexpr int SB = 32;
constexpr int SB_THREADS = 128;

__global__ void __launch_bounds__(SB_THREADS) gemm_f64_s32_kernel(int64_t M, int64_t N, int64_t K,
                                                                  double alpha,
                                                                  const double *__restrict__ A,
                                                                  int64_t lda, int opA,
                                                                  const double *__restrict__ B,
                                                                  int64_t ldb, int opB, double beta,
                                                                  double *C, int64_t ldc,
                                                                  F64Mask mask,
                                                                  const int64_t *info) {
    __shared__ double As[GBK][SB + 1];
    __shared__ double Bs[GBK][SB + 1];
    if (info && failed(info)) return;
    const int64_t r0 = (int64_t)blockIdx.x * SB, c0 = (int64_t)blockIdx.y * SB;
    if (mask.out_lower && c0 > r0 + (SB - 1) + mask.diag_off) return;
    int64_t kbeg = 0, kend = K;
    if (mask.kchunk > 0) {
        kbeg = (int64_t)blockIdx.z * mask.kchunk;
        kend = min(K, kbeg + mask.kchunk);
    }
    if (mask.tri_k && c0 - mask.tri_off > kbeg) kbeg = ((c0 - mask.tri_off) / GBK) * GBK;
    if (kbeg >= kend) return;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;  // rows tx + 16a (a < 2), columns ty + 8b (b < 4)
    double acc[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + SB_THREADS * q;  // 0..511
            int r, k, c, kb;
            double v = 0.0, w = 0.0;
            if (opA == 0) { r = idx & 31; k = idx >> 5; }
            else { k = idx & 15; r = idx >> 4; }
            {
                const int64_t gr = r0 + r, gk = k0 + k;
                if (gr < M && gk < kend) v = opA == 0 ? A[gr + gk * lda] : A[gk + gr * lda];
            }
            As[k][r] = v;
            if (opB == 0) { kb = idx & 15; c = idx >> 4; }
            else { c = idx & 31; kb = idx >> 5; }
            {
                const int64_t gc = c0 + c, gk = k0 + kb;
                if (gc < N && gk < kend) w = opB == 0 ? B[gk + gc * ldb] : B[gc + gk * ldb];
            }
            Bs[kb][c] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GBK; ++k) {
            double av[2], bv[4];
#pragma unroll
            for (int a = 0; a < 2; ++a) av[a] = As[k][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[k][ty + 8 * b];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int64_t gc = c0 + ty + 8 * b;
        if (gc >= N) continue;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int64_t gr = r0 + tx + 16 * a;
            if (gr >= M) continue;
            if (mask.out_lower && gr + mask.diag_off < gc) continue;
            double *p = C + gr + gc * ldc;
            if (mask.kchunk > 0) {
                atomicAdd(p, alpha * acc[a][b]);
            } else {
                double v = alpha * acc[a][b];
                if (beta != 0.0) v = fma(beta, *p, v);
                *p = v;
            }
        }
    }
}

int gemm_f64_ex(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
                int opA, const double *B, int64_t ldb, int opB, double beta, double *C, int64_t ldc,
                int lower, const F64Mask &mask, const int64_t *info, cudaStream_t s) {
    if (M <= 0 || N <= 0) return GP_OK;
    const int64_t tiles64 = lower ? ceil_div(M, TB) * (ceil_div(M, TB) + 1) / 2
                                  : ceil_div(M, TB) * ceil_div(N, TB);
    if (mask.kchunk > 0 || tiles64 < 256) {
        // small launch: 32 x 32 tiles (a lower request masks the upper tiles)
        F64Mask m = mask;
        if (lower) {
            m.out_lower = 1;
            m.diag_off = 0;
        }
        if (m.kchunk > 0 && beta != 1.0) {
            if (beta != 0.0) return GP_ERR_INVALID;  // split K accumulates into C
        }
        const int64_t kz = m.kchunk > 0 ? ceil_div(K, m.kchunk) : 1;
        dim3 g((unsigned)ceil_div(M, SB), (unsigned)ceil_div(N, SB), (unsigned)kz);
        gemm_f64_s32_kernel<<<g, SB_THREADS, 0, s>>>(M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc,
                                             m, info);
        GP_LAUNCH_CHECK();
        return GP_OK;
    }
    if (lower) {
        if (M != N) return GP_ERR_INVALID;
        int64_t T = ceil_div(M, TB);
        gemm_f64_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(
            M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc, 1, mask, info);
    } else {
        dim3 g((unsigned)ceil_div(M, TB), (unsigned)ceil_div(N, TB));
        gemm_f64_kernel<<<g, 256, 0, s>>>(M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc, 0,
                                          mask, info);
    }
    GP_LAUNCH_CHECK();
    return GP_OK;
}

int gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda, int opA,
             const double *B, int64_t ldb, int opB, double beta, double *C, int64_t ldc, int lower,
             const int64_t *info, cudaStream_t s) {
    F64Mask none{0, 0, 0, 0, 0};
    return gemm_f64_ex(M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc, lower, none, info, s);
}

// ---------------------------------------------------------------------------
// Right-looking tiled Cholesky in FP64 of the m x m block at A (m a multiple
// of 64): per tile column k, POTRF of the diagonal tile, TRSM of the tiles
// below, SYRK/GEMM of the trailing lower triangle (Sec. 2.1).
// ---------------------------------------------------------------------------
int chol_fp64_tiled(double *A, int64_t ld, int64_t m, int64_t col_base, int64_t *info,
                    cudaStream_t s) {
    const int64_t T = m / TB;
    for (int64_t k = 0; k < T; ++k) {
        const int64_t k0 = k * TB;
        double *Akk = A + k0 + k0 * ld;
        potrf_tile_kernel<<<1, 256, 0, s>>>(Akk, ld, col_base + k0, info);
        GP_LAUNCH_CHECK();
        const int64_t rest = m - k0 - TB;
        if (rest <= 0) continue;
        double *P = Akk + TB;  // rows below the diagonal tile
        trsm_tiles_kernel<<<(unsigned)ceil_div(rest, TR_ROWS), 256, 0, s>>>(Akk, P, ld, rest, info);
        GP_LAUNCH_CHECK();
        double *C = P + TB * ld;  // trailing block
        GP_TRY(gemm_f64(rest, rest, TB, -1.0, P, ld, 0, P, ld, 1, 1.0, C, ld, 1, info, s));
    }
    return GP_OK;
}

// ---------------------------------------------------------------------------
// X = L^{-1} for the lower m x m block L (m a multiple of 64), FP64, written
// to X (ld_x; full block, zeros above the diagonal).  Block forward
// substitution over 64-row tiles: X_ii = L_ii^{-1};
// X_{i,0:i} = -X_ii (L_{i,0:i} X_{0:i,0:i}).  tmp: 64 x m doubles.
// ---------------------------------------------------------------------------
int trtri_fp64_blocked(const double *L, int64_t ld_l, int64_t m, double *X, int64_t ld_x,
                       double *tmp, const int64_t *info, cudaStream_t s) {
    const int64_t T = m / TB;
    if (cudaMemset2DAsync(X, ld_x * sizeof(double), 0, m * sizeof(double), m, s) != cudaSuccess)
        return GP_ERR_CUDA;
    trtri_tiles_kernel<<<(unsigned)T, 256, 0, s>>>(L, ld_l, X, ld_x, info);
    GP_LAUNCH_CHECK();
    for (int64_t i = 1; i < T; ++i) {
        const int64_t i0 = i * TB;
        // tmp (64 x i0) = L[i0:i0+64, 0:i0] * X[0:i0, 0:i0]; X lower, so column
        // block j needs K >= j only; K split in 64-chunks accumulated atomically
        if (cudaMemsetAsync(tmp, 0, sizeof(double) * TB * i0, s) != cudaSuccess) return GP_ERR_CUDA;
        F64Mask split{0, 0, 1, 0, TB};
        GP_TRY(gemm_f64_ex(TB, i0, i0, 1.0, L + i0, ld_l, 0, X, ld_x, 0, 1.0, tmp, TB, 0, split,
                           info, s));
        // X[i0:i0+64, 0:i0] = -X_ii * tmp
        GP_TRY(gemm_f64(TB, i0, TB, -1.0, X + i0 + i0 * ld_x, ld_x, 0, tmp, TB, 0, 0.0, X + i0,
                        ld_x, 0, info, s));
    }
    return GP_OK;
}

}  // namespace gp
