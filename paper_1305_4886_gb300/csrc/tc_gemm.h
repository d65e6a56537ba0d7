// tc_gemm.h -- BF16-slice tensor-core contraction (tcgen05) interface.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gp {

// A packed operand: bf16 slices [S][rows][K], K contiguous.  row_off selects
// the first operand row used by a contraction.
struct TcOperand {
    const __nv_bfloat16 *slices;
    int64_t rows;
    int64_t K;
    int S;
    int64_t row_off;
};

struct TcGemmArgs {
    double *C;
    int64_t ldc;
    int64_t M, N;
    double alpha, beta;
    int kblocks;
    int npairs;
    int pa[16], pb[16];
    int lower;
    int a_row_off, b_row_off;
    int64_t *info;
};

// C (M x N, column-major FP64) = beta C + alpha sum_{p+q<S} A_p B_q^T, where
// A_p / B_q are the slices of the packed operands (M / N rows, K columns).
// lower != 0: only entries with row >= col are written (C's diagonal on the
// operand diagonal).
int tc_gemm(const TcOperand &A, const TcOperand &B, int64_t M, int64_t N, int64_t K, double alpha,
            double beta, double *C, int64_t ldc, int lower, int nslices, int64_t *info,
            cudaStream_t s);

// Pack src (R x Kvalid, see split_bf16_kernel for trans / lower_mask) into S
// bf16 slices dst[S][R][K], zero-padded to K columns.
int split_bf16(const double *src, int64_t ld, int64_t R, int64_t K, int64_t Kvalid, int trans,
               int64_t diag_off, int lower_mask, int S, __nv_bfloat16 *dst, cudaStream_t s);

}  // namespace gp
