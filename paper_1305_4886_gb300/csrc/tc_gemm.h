// tc_gemm.h -- BF16-slice tensor-core contraction (tcgen05) interface.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gp {

// A packed operand store: bf16 slices [S][rows][Kld] (K contiguous, Kld a
// multiple of 64).  A contraction reads rows row_off.. and K columns
// k_off.. (k_off a multiple of 64).
struct TcOperand {
    const __nv_bfloat16 *slices;
    int64_t rows;
    int64_t Kld;
    int S;
    int64_t row_off;
    int64_t k_off;
};

// Output of a contraction.  fp32 = 0: C is FP64, C = beta C + alpha acc;
// fp32 = 1: C is FP32, C += alpha acc.  lower: write only entries with
// row + diag_off >= col (local coordinates).
struct TcOut {
    void *C;
    int64_t ldc;
    int fp32;
    double alpha;
    double beta;
    int lower;
    int64_t diag_off;
};

// out(M x N) <- sum over slice pairs p + q < S of A_p B_q^T, K columns.
// tri_k != 0: B(k, c) is known to vanish for k < c - tri_off, so each tile
// starts its K loop at its first column minus tri_off (rounded down to 64).
int tc_gemm(const TcOperand &A, const TcOperand &B, int64_t M, int64_t N, int64_t K,
            const TcOut &out, int tri_k, int64_t tri_off, int64_t *info, cudaStream_t s);

// Pack src (R x K region; see split_rows_kernel for trans / lower_mask) into
// S row-scaled slices at dst[p][dst_row_off + r][dst_k_off + k] of a store
// with dst_rows rows and dst_kld columns.  Columns k >= Kvalid are zero.
int split_rows(const double *src, int64_t ld, int64_t R, int64_t K, int64_t Kvalid, int trans,
               int64_t diag_off, int lower_mask, int S, __nv_bfloat16 *dst, int64_t dst_rows,
               int64_t dst_kld, int64_t dst_row_off, int64_t dst_k_off, cudaStream_t s);

}  // namespace gp
