// tc_gemm.h -- 16-bit-slice tensor-core contraction (tcgen05) interface.
#pragma once

#include "common.cuh"

namespace gp {

constexpr int64_t TC_CHUNK_K = 512;  // K depth of one row bound / exact chunk

// A packed operand store: 16-bit slices [S][rows][Kld] (K contiguous, Kld a
// multiple of 64).  A contraction reads rows row_off.. and K columns
// k_off.. (k_off a multiple of 64).  Two encodings, by slice count:
//   S = 3 (mixed form), normalized: FP16 values of x 2^{7 - e}, with
//     e = ex[row * ex_ld + k / 512] the bound exponent of the row over each
//     512-deep chunk of K: s0 an integer in [-128, 128], s1 and s2 the FP16
//     roundings of the remainders.  The contraction scales each chunk's
//     sums by 2^{e_a + e_b - 14} in its epilogue.
//   S = 5 (FP64-grade form), scaled: BF16 values q_p 2^{e - 7 - 8p}, q_p an
//     integer in [-128, 128]; ex is unused.
struct TcOperand {
    const uint16_t *slices;
    int64_t rows;
    int64_t Kld;
    int S;
    int64_t row_off;
    int64_t k_off;
    const int *ex = nullptr;
    int64_t ex_ld = 0;
    int64_t kch = TC_CHUNK_K;  // K width of one row bound (512, or 1024 for a
                               // three-slice store packed with wider chunks)
};

// Exponent columns of a store with Kld columns and row bounds per kch columns.
inline int64_t tc_ex_ld(int64_t Kld, int64_t kch = TC_CHUNK_K) { return (Kld + kch - 1) / kch; }

// Output of a contraction.  mode 0: C is FP64, C = beta C + alpha acc;
// mode 2: C is an FP32 pair (float2 hi, lo) updated in double-float
// arithmetic, C += alpha acc.  lower: write only
// entries with row + diag_off >= col (local coordinates).
struct TcOut {
    void *C;
    int64_t ldc;
    int mode;
    double alpha;
    double beta;
    int lower;
    int64_t diag_off;
    void *acc2 = nullptr;  // mode 0 with K > 512: M x N float2 scratch; the
                           // accumulators are flushed per 512-deep chunk into it
                           // in double-float and converted to FP64 at the end
    int max_ctas = 0;      // > 0: at most this many persistent CTAs (leaves the
                           // other SMs to work on another stream)
};

// out(M x N) <- sum over slice pairs p + q < S of A_p B_q^T, K columns.
// K > 512 is accumulated per 512-deep chunk (mode 2 directly, mode 0 through
// acc2, which it then requires); operand k_off must be multiples of 512.
// tri_k != 0: B(k, c) is known to vanish for k < c - tri_off, so each tile
// starts its K loop at its first column minus tri_off (rounded down to 64).
int tc_gemm(const TcOperand &A, const TcOperand &B, int64_t M, int64_t N, int64_t K,
            const TcOut &out, int tri_k, int64_t tri_off, int64_t *info, cudaStream_t s);

// Pack src (R x K region; see split_rows_kernel for trans / lower_mask) into
// S row-scaled slices at dst[p][dst_row_off + r][dst_k_off + k] of a store
// with dst_rows rows and dst_kld columns (dst_k_off a multiple of 512).
// Columns k >= Kvalid are zero.  S = 3 also writes the row exponents to
// dst_ex (dst_rows x tc_ex_ld(dst_kld) ints).
// kch: K width of one row bound (512; 1024 allowed for three slices, where
// group 0 stays exact in FP32 for K <= 1024).
int split_rows(const double *src, int64_t ld, int64_t R, int64_t K, int64_t Kvalid, int trans,
               int64_t diag_off, int lower_mask, int S, uint16_t *dst, int *dst_ex,
               int64_t dst_rows, int64_t dst_kld, int64_t dst_row_off, int64_t dst_k_off,
               cudaStream_t s, int64_t kch = TC_CHUNK_K);

}  // namespace gp
