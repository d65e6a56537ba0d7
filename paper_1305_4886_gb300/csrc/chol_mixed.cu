// chol_mixed.cu -- mixed-precision blocked Cholesky (Sec. 2.1 block
// algorithm, two levels of blocking as in Sec. 2.2).
//
// Outer blocks of NB = 512 columns.  Per outer block column k:
//   1. FP64 tiled Cholesky of the NB x NB diagonal block (64-column tiles,
//      diagonal POTRF in shared memory)                       -- FP64
//   2. W = L_kk^{-1} by blocked FP64 triangular inversion       -- FP64
//   3. panel solve L_ik = A_ik W^T as one tensor-core contraction over
//      BF16 slices of A_ik and W (the forward-solves of Sec. 2.1)
//   4. trailing update A_ij -= L_ik L_jk^T for the lower triangle, on the
//      tensor cores over BF16 slices of the panel ("most of the total work
//      is in the matrix multiplications", Sec. 2.1).
// The diagonal pivots, hence the log-determinant, come from FP64
// factorisations of blocks that carry FP32-accurate updates.
#include "internal.h"
#include "tc_gemm.h"

namespace gp {

constexpr int64_t NB = 512;

struct MixedWs {
    double *W = nullptr;            // NB x NB, inverse of the diagonal block
    double *tmp = nullptr;          // 64 x NB
    __nv_bfloat16 *SA = nullptr;    // S x np x NB  panel slices
    __nv_bfloat16 *SB = nullptr;    // S x NB x NB  inverse slices
    size_t bytes = 0;
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static MixedWs mixed_layout(void *base, int64_t np, int S) {
    MixedWs w;
    char *b = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = align256(off);
        char *p = b ? b + off : nullptr;
        off += bytes;
        return p;
    };
    w.W = reinterpret_cast<double *>(take(sizeof(double) * NB * NB));
    w.tmp = reinterpret_cast<double *>(take(sizeof(double) * TB * NB));
    w.SA = reinterpret_cast<__nv_bfloat16 *>(take(2ull * S * (size_t)np * NB));
    w.SB = reinterpret_cast<__nv_bfloat16 *>(take(2ull * S * NB * NB));
    w.bytes = align256(off);
    return w;
}

size_t chol_mixed_ws_bytes(int64_t np, int S) { return mixed_layout(nullptr, np, S).bytes; }

int chol_mixed(double *A, int64_t ld, int64_t np, int S, void *ws, int64_t *info, cudaStream_t s) {
    MixedWs w = mixed_layout(ws, np, S);
    for (int64_t k0 = 0; k0 < np; k0 += NB) {
        const int64_t nb = (np - k0) < NB ? (np - k0) : NB;
        double *Akk = A + k0 + k0 * ld;
        GP_TRY(chol_fp64_tiled(Akk, ld, nb, k0, info, s));
        const int64_t m = np - k0 - nb;
        if (m <= 0) break;
        double *P = Akk + nb;  // m x nb panel below the diagonal block
        GP_TRY(trtri_fp64_blocked(Akk, ld, nb, w.W, nb, w.tmp, info, s));
        GP_TRY(split_bf16(w.W, nb, nb, nb, nb, 0, 0, 0, S, w.SB, s));
        GP_TRY(split_bf16(P, ld, m, nb, nb, 0, 0, 0, S, w.SA, s));
        TcOperand opA{w.SA, m, nb, S, 0};
        TcOperand opW{w.SB, nb, nb, S, 0};
        // L_ik = A_ik W^T
        GP_TRY(tc_gemm(opA, opW, m, nb, nb, 1.0, 0.0, P, ld, 0, S, info, s));
        GP_TRY(split_bf16(P, ld, m, nb, nb, 0, 0, 0, S, w.SA, s));
        // A_22 -= L_ik L_ik^T (lower)
        GP_TRY(tc_gemm(opA, opA, m, m, nb, -1.0, 1.0, P + nb * ld, ld, 1, S, info, s));
    }
    return GP_OK;
}

// ---------------------------------------------------------------------------
// Standalone trailing update C (m x m, lower) -= P P^T, P m x k.
// ---------------------------------------------------------------------------
size_t syrk_ws_bytes(int64_t m, int64_t k, int precision, int S) {
    if (precision == GP_FP64) return 0;
    return align256(2ull * S * (size_t)m * (size_t)round_up(k, 64));
}

int syrk_lower(double *C, int64_t ldc, const double *P, int64_t ldp, int64_t m, int64_t k,
               int precision, int S, void *ws, int64_t *info, cudaStream_t s) {
    if (precision == GP_FP64)
        return gemm_f64(m, m, k, -1.0, P, ldp, 0, P, ldp, 1, 1.0, C, ldc, 1, info, s);
    __nv_bfloat16 *SA = static_cast<__nv_bfloat16 *>(ws);
    const int64_t kp = round_up(k, 64);
    GP_TRY(split_bf16(P, ldp, m, kp, k, 0, 0, 0, S, SA, s));
    TcOperand op{SA, m, kp, S, 0};
    return tc_gemm(op, op, m, m, kp, -1.0, 1.0, C, ldc, 1, S, info, s);
}

}  // namespace gp
