// dense_f64.cu -- FP64 CUDA-core building blocks of the tiled Cholesky
// (Sec. 2.1: factor the diagonal block, forward-solve the blocks below it,
// update the trailing blocks by multiply-and-subtract; repeat per block
// column).
//
//   potrf_tile   Cholesky of one 64 x 64 diagonal tile in shared memory,
//                blocked by 8 columns.
//   trsm_tiles   panel solve  B <- B L_kk^{-T}  for the tiles below it.
//   trtri_tiles  inverse of each 64 x 64 diagonal tile of a lower block.
//   gemm_f64     C = alpha op(A) op(B) + beta C, 64 x 64 register-tiled.
//
// GB300 executes FP64 at a small fraction of its tensor rate, so these
// kernels are bounded by the FP64 pipe, not by memory: a 4 x 4 register tile
// per thread keeps shared-memory traffic far below the DFMA issue rate.
#include "internal.h"
#include "kern_df.cuh"

namespace gp {

// ---------------------------------------------------------------------------
// Cholesky of the 64 x 64 tile at A (column-major, ld) in shared memory, on
// the unscaled columns: a_rc -= a_rj a_cj / d_j (d_j the current pivot),
// the columns scaled by 1/sqrt(d_j) once at the end (L_rj = a_rj /
// sqrt(d_j)).  Blocked by PB columns: one warp factors a panel of PB columns
// (all rows below them; only warp synchronisation between its columns),
// then every thread applies the panel's PB updates to its entries of the
// trailing lower triangle (PB FMAs per index computation).  Two block
// barriers per panel instead of two per column: on this part the per-column
// barriers and dependency latencies, not the FP64 pipe, bounded the
// column-at-a-time form (66 us per tile against about 20 us of FP64 work).
// col_base is the global column of the tile's first column (for the d_info
// convention).  A pivot <= 0 or NaN stops the factorisation.
// ---------------------------------------------------------------------------
constexpr int PB = 8;

__global__ void __launch_bounds__(256) potrf_tile_kernel(double *A, int64_t ld, int64_t col_base,
                                                         int64_t *info) {
    __shared__ double S[TB * (TB + 1)];
    __shared__ double lj[PB][TB];  // a_cj / d_j: panel column j, trailing column c
    __shared__ double dinv[TB];
    __shared__ int bad;
    if (failed(info)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        S[c * (TB + 1) + r] = (r >= c) ? A[r + (int64_t)c * ld] : 0.0;
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int p = 0; p < TB; p += PB) {
        if (warp == 0) {
            // panel columns p .. p + PB - 1 (rows c .. 63 of each column c)
            for (int j = p; j < p + PB; ++j) {
                const double *cj = S + j * (TB + 1);
                const double d = cj[j];
                if (!(d > 0.0)) {  // every lane read the same pivot
                    if (lane == 0) {
                        bad = 1;
                        set_info(info, col_base + j + 1);
                    }
                    break;
                }
                const double inv = 1.0 / d;
                if (lane == 0) dinv[j] = inv;
                for (int c = j + 1; c < p + PB; ++c) {
                    const double l = cj[c] * inv;
                    double *cc = S + c * (TB + 1);
                    for (int r = c + lane; r < TB; r += 32) cc[r] = fma(-cj[r], l, cc[r]);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (bad) break;  // uniform
        const int q = p + PB;  // first trailing column
        if (q >= TB) break;
        const int nt = TB - q;
        for (int e = tid; e < PB * nt; e += blockDim.x) {
            const int jj = e / nt, c = q + e % nt;
            lj[jj][c] = S[(p + jj) * (TB + 1) + c] * dinv[p + jj];
        }
        __syncthreads();
        // trailing lower triangle q <= c <= r < 64
        const int ntri = nt * (nt + 1) / 2;
        for (int e = tid; e < ntri; e += blockDim.x) {
            int r, c;
            tri_desc_entry(e, nt, r, c);
            r += q;
            c += q;
            double acc = S[c * (TB + 1) + r];
#pragma unroll
            for (int jj = 0; jj < PB; ++jj) acc = fma(-S[(p + jj) * (TB + 1) + r], lj[jj][c], acc);
            S[c * (TB + 1) + r] = acc;
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
// The same blocked factorisation in double-float arithmetic (pairs of FP32
// numbers, about 48 significant bits) on the FP32 pipe, for the diagonal
// blocks of the tensor-core forms, whose inputs (the FP64 matrix plus the
// double-float pending updates) carry no more.  On this part a dependent
// FP64 FMA takes about 47 cycles and an FP64 division about 540, against
// about 4 for an FP32 operation, and the column chain of the factorisation
// (pivot reciprocal, multipliers, update, next pivot) is latency bound.  The
// tile is converted from FP64 by integer operations and written back in FP64.
// ---------------------------------------------------------------------------
// One PB-column panel of potrf_tile_df_kernel, on one warp, in registers:
// the lane owns rows lane and lane + 32 of the panel's columns; pivots and
// multipliers travel by shuffles (entries above a column's diagonal are
// updated too, and never read).  The panel's own rows lie in row slot SLOT.
template <int SLOT>
__device__ __forceinline__ void df_panel(dfl *S, dfl *dinv, int *bad, int p, int lane,
                                         int64_t col_base, int64_t *info) {
    float vh[2][PB], vl[2][PB];  // the pairs' high and low parts, kept apart (registers)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < PB; ++jj) {
            const dfl x = S[(p + jj) * (TB + 1) + lane + 32 * i];
            vh[i][jj] = x.h;
            vl[i][jj] = x.l;
        }
    bool ok = true;
#pragma unroll
    for (int jj = 0; jj < PB; ++jj) {
        const int j = p + jj;
        const dfl d{__shfl_sync(0xffffffffu, vh[SLOT][jj], j & 31),
                    __shfl_sync(0xffffffffu, vl[SLOT][jj], j & 31)};
        if (ok && !(d.h > 0.0f)) {  // uniform; the first failing pivot is reported
            if (lane == 0) {
                *bad = 1;
                set_info(info, col_base + j + 1);
            }
            ok = false;
        }
        const dfl inv = df_rcp(d);
        if (lane == 0) dinv[j] = inv;
        // a constant trip count (the guard folds once both loops are
        // unrolled), so that every register index is static
#pragma unroll
        for (int cc = 1; cc < PB; ++cc) {
            if (cc <= jj) continue;
            const int c = p + cc;
            const dfl l = df_mul(dfl{__shfl_sync(0xffffffffu, vh[SLOT][jj], c & 31),
                                     __shfl_sync(0xffffffffu, vl[SLOT][jj], c & 31)},
                                 inv);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const dfl r = df_fms(dfl{vh[i][cc], vl[i][cc]}, dfl{vh[i][jj], vl[i][jj]}, l);
                vh[i][cc] = r.h;
                vl[i][cc] = r.l;
            }
        }
    }
    if (ok) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int jj = 0; jj < PB; ++jj)
                S[(p + jj) * (TB + 1) + lane + 32 * i] = dfl{vh[i][jj], vl[i][jj]};
    }
}

__global__ void __launch_bounds__(256) potrf_tile_df_kernel(double *A, int64_t ld,
                                                            int64_t col_base, int64_t *info) {
    __shared__ dfl S[TB * (TB + 1)];
    __shared__ dfl lj[PB][TB];  // a_cj / d_j: panel column j, trailing column c
    __shared__ dfl dinv[TB];
    __shared__ int bad;
    if (failed(info)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        S[c * (TB + 1) + r] =
            (r >= c) ? f64_to_df(static_cast<unsigned long long>(
                           __double_as_longlong(A[r + (int64_t)c * ld])))
                     : dfl{0.0f, 0.0f};
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int p = 0; p < TB; p += PB) {
        if (warp == 0) {
            if (p < 32)
                df_panel<0>(S, dinv, &bad, p, lane, col_base, info);
            else
                df_panel<1>(S, dinv, &bad, p, lane, col_base, info);
        }
        __syncthreads();
        if (bad) break;  // uniform
        const int q = p + PB;
        if (q >= TB) break;
        const int nt = TB - q;
        for (int e = tid; e < PB * nt; e += blockDim.x) {
            const int jj = e / nt, c = q + e % nt;
            lj[jj][c] = df_mul(S[(p + jj) * (TB + 1) + c], dinv[p + jj]);
        }
        __syncthreads();
        const int ntri = nt * (nt + 1) / 2;
        for (int e = tid; e < ntri; e += blockDim.x) {
            int r, c;
            tri_desc_entry(e, nt, r, c);
            r += q;
            c += q;
            dfl acc = S[c * (TB + 1) + r];
#pragma unroll
            for (int jj = 0; jj < PB; ++jj) acc = df_fms(acc, S[(p + jj) * (TB + 1) + r], lj[jj][c]);
            S[c * (TB + 1) + r] = acc;
        }
        __syncthreads();
    }
    if (bad) return;
    if (tid < TB) dinv[tid] = df_sqrt(dinv[tid]);
    __syncthreads();
    for (int e = tid; e < TB * TB; e += blockDim.x) {
        int r = e & (TB - 1), c = e >> 6;
        if (r >= c) A[r + (int64_t)c * ld] = df_to_double(df_mul(S[c * (TB + 1) + r], dinv[c]));
    }
}

// ---------------------------------------------------------------------------
// B <- B L^{-T} for the rows below the diagonal tile L (the panel
// forward-solve of Sec. 2.1).  Each CTA solves 16 rows (rows r0 = 16 blockIdx
// of B0) against the whole 64 x 64 triangle (more CTAs for the latency-bound
// small panels of the diagonal blocks); the pivots' reciprocals are formed
// once.
// ---------------------------------------------------------------------------
constexpr int TR_ROWS = 16;

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
        int r = e & (TR_ROWS - 1), c = e / TR_ROWS;
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
        int r = e & (TR_ROWS - 1), c = e / TR_ROWS;
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
// mask.a_lower: op(A) is lower triangular (op(A)(r, k) = 0 for k > r, the
// upper part never read); tiles end their K loop after their last row.
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
    const int64_t kend = mask.a_lower ? min(K, r0 + TB) : K;  // op(A) lower: k <= r
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int idx = tid + 256 * q;
            int r, k;
            double v = 0.0;
            if (opA == 0) {
                r = idx & 63;
                k = idx >> 6;
                int64_t gr = r0 + r, gk = k0 + k;
                if (gr < M && gk < K && (!mask.a_lower || gk <= gr)) v = A[gr + gk * lda];
            } else {
                k = idx & 15;
                r = idx >> 4;
                int64_t gr = r0 + r, gk = k0 + k;
                if (gr < M && gk < K && (!mask.a_lower || gk <= gr)) v = A[gk + gr * lda];
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
// grid.z and adds each partial product with FP64 atomics: C += alpha A B
// (beta must be 1; kchunk a multiple of GBK).
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
    if (mask.a_lower) kend = min(kend, r0 + SB);  // op(A) lower: k <= r
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
                if (gr < M && gk < kend && (!mask.a_lower || gk <= gr))
                    v = opA == 0 ? A[gr + gk * lda] : A[gk + gr * lda];
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
        // split K adds every chunk's partial product into C: only C += alpha op(A) op(B)
        // is expressible, and chunks must start on the kernel's 16-deep K steps (the
        // triangular start is rounded down to one)
        if (m.kchunk > 0 && (beta != 1.0 || m.kchunk % GBK != 0)) return GP_ERR_INVALID;
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
// below, SYRK/GEMM of the trailing lower triangle (Sec. 2.1).  df_tiles:
// the diagonal tiles are factored in double-float (potrf_tile_df_kernel).
// ---------------------------------------------------------------------------
int chol_fp64_tiled(double *A, int64_t ld, int64_t m, int64_t col_base, int64_t *info,
                    cudaStream_t s, bool df_tiles) {
    const int64_t T = m / TB;
    for (int64_t k = 0; k < T; ++k) {
        const int64_t k0 = k * TB;
        double *Akk = A + k0 + k0 * ld;
        if (df_tiles)
            potrf_tile_df_kernel<<<1, 256, 0, s>>>(Akk, ld, col_base + k0, info);
        else
            potrf_tile_kernel<<<1, 256, 0, s>>>(Akk, ld, col_base + k0, info);
        GP_LAUNCH_CHECK();
        const int64_t rest = m - k0 - TB;
        if (rest <= 0) continue;
        double *P = Akk + TB;  // rows below the diagonal tile
        trsm_tiles_kernel<<<(unsigned)ceil_div(rest, TR_ROWS), 256, 0, s>>>(Akk, P, ld, rest, info);
        GP_LAUNCH_CHECK();
        double *C = P + TB * ld;  // trailing block
        // small (latency-bound) updates: K = 64 split in four over the grid
        // (FP64 atomics into C), four times the CTAs
        F64Mask split{0, 0, 0, 0, rest <= 512 ? 16 : 0};
        GP_TRY(gemm_f64_ex(rest, rest, TB, -1.0, P, ld, 0, P, ld, 1, 1.0, C, ld, 1, split, info, s));
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
        // block j needs K >= j only.  Both products are small and latency
        // bound: K is split in 16-chunks over the grid, accumulated atomically
        if (cudaMemsetAsync(tmp, 0, sizeof(double) * TB * i0, s) != cudaSuccess) return GP_ERR_CUDA;
        F64Mask split{0, 0, 1, 0, 16};
        GP_TRY(gemm_f64_ex(TB, i0, i0, 1.0, L + i0, ld_l, 0, X, ld_x, 0, 1.0, tmp, TB, 0, split,
                           info, s));
        // X[i0:i0+64, 0:i0] = -X_ii * tmp, into the zeros set above
        F64Mask k16{0, 0, 0, 0, 16};
        GP_TRY(gemm_f64_ex(TB, i0, TB, -1.0, X + i0 + i0 * ld_x, ld_x, 0, tmp, TB, 0, 1.0, X + i0,
                           ld_x, 0, k16, info, s));
    }
    return GP_OK;
}

}  // namespace gp
