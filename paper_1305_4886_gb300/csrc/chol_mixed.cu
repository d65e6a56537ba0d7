// chol_mixed.cu -- mixed-precision blocked Cholesky (the block algorithm of
// Sec. 2.1 with the two levels of blocking of Sec. 2.2).
//
// Outer blocks of NB = 512 columns.  The matrix stays FP64 (the fill's C);
// trailing updates accumulate in a separate double-float array D (FP32
// pairs hi + lo, about 48 significant bits, updated with FP32 error-free
// sums) that is folded into the FP64 matrix one block column at a time, just
// before that column is factored, so the FP64 pipe (1/64 of the FP32 rate on
// this part) touches each entry once instead of once per outer step.  An
// FP32 D would round every pending entry once per outer step, a relative
// error growing like 2^-24 sqrt(n / NB).  Per outer block column k:
//   1. A[k:, k] += D[k:, k]   (FP64 += hi + lo, the block column only)
//   2. FP64 tiled Cholesky of the NB x NB diagonal block      -- FP64
//   3. W = L_kk^{-1}, blocked FP64 triangular inversion        -- FP64
//   4. panel solve L_ik = A_ik W^T: one tensor-core contraction over row-
//      scaled BF16 slices of A_ik and W (the forward-solves of Sec. 2.1),
//      written to the FP64 matrix
//   5. trailing update D_ij -= L_ik L_jk^T on the lower triangle, tensor
//      cores, double-float accumulation into D ("most of the total work is
//      in the matrix multiplications", Sec. 2.1).
// Lookahead: step 5 updates block column k+1 first; steps 1-3 of block k+1
// then run on a side stream (on the few SMs the rest of the update leaves
// free) while the rest of step 5 runs, so the latency-bound diagonal
// blocks leave the critical path (the paper's diagonal blocks are likewise
// the sequential part of each step, Sec. 2.1).
// The pivots and hence the log-determinant come from FP64 factorisations of
// blocks whose updates carry the slice products' accuracy.
#include <stdlib.h>

#include <mutex>

#include "internal.h"
#include "kern_df.cuh"
#include "tc_gemm.h"

namespace gp {

constexpr int64_t NB_MAX = 512;

// Outer block width, 512 columns in both tensor-core forms.  Measured and not
// kept: 1024-column blocks with the trailing update's row bounds over 1024
// columns (4% faster over the headline step, 10x less accurate in the
// log-determinant, gradient 1.5e-6 at n = 16,384), and 1024-column blocks
// with 512-column row bounds (the update flushed twice per tile: as
// accurate, 3% slower).
int64_t chol_block_cols(int) { return NB_MAX; }

struct MixedWs {
    double *W = nullptr;            // NB x NB, inverse of the diagonal block
    double *tmp = nullptr;          // 64 x NB
    uint16_t *SA = nullptr;         // S x np x NB  panel slices
    uint16_t *SB = nullptr;         // S x NB x NB  inverse slices
    int *exA = nullptr, *exB = nullptr;  // their row exponents (three-slice form)
    float2 *D = nullptr;            // np x np pending trailing updates (double-float)
    int64_t np = 0;
    size_t bytes = 0;
};

static int64_t np_of(const MixedWs &w) { return w.np; }

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static MixedWs mixed_layout(void *base, int64_t np, int S) {
    MixedWs w;
    const int64_t NB = NB_MAX;  // sized for the widest block
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
    w.SA = reinterpret_cast<uint16_t *>(take(2ull * S * (size_t)np * NB));
    w.SB = reinterpret_cast<uint16_t *>(take(2ull * S * NB * NB));
    w.exA = reinterpret_cast<int *>(take(sizeof(int) * (size_t)np * tc_ex_ld(NB, 512)));
    w.exB = reinterpret_cast<int *>(take(sizeof(int) * NB * tc_ex_ld(NB, 512)));
    w.D = reinterpret_cast<float2 *>(take(sizeof(float2) * (size_t)np * (size_t)np));
    w.np = np;
    w.bytes = align256(off);
    return w;
}

size_t chol_mixed_ws_bytes(int64_t np, int S) { return mixed_layout(nullptr, np, S).bytes; }

size_t chol_winv_doubles(int64_t np) { return (size_t)ceil_div(np, NB_MAX) * NB_MAX * NB_MAX; }

// The inverse of the 512-column diagonal block at k0 inside the stored
// inverses of the factorisation's diagonal blocks (blocks of
// chol_block_cols(S) columns, each stored with ld = its width): a diagonal
// sub-block of a block's inverse is the sub-block's inverse.
const double *winv_block(const double *winv, int64_t np, int S, int64_t k0, int64_t *ld) {
    const int64_t NB = chol_block_cols(S);
    const int64_t q0 = (k0 / NB) * NB;
    const int64_t w = (np - q0) < NB ? (np - q0) : NB;
    const int64_t off = k0 - q0;
    *ld = w;
    return winv + (q0 / NB) * NB * NB + off + off * w;
}

// A[r, c] += D.hi[r, c] + D.lo[r, c] (double-float pending updates) for the
// lower entries r + roff >= c of a rows x cols block.
__global__ void fold_delta2_kernel(double *A, int64_t ld, const float2 *D, int64_t ldd,
                                   int64_t rows, int64_t cols, int64_t roff, const int64_t *info) {
    if (failed(info)) return;
    const int64_t c = blockIdx.y;
    const int64_t rfirst = c - roff > 0 ? c - roff : 0;
    for (int64_t r = rfirst + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const float2 d = D[r + c * ldd];
        A[r + c * ld] += f32_to_f64(d.x) + f32_to_f64(d.y);  // conversions by integer operations
    }
}

// Lookahead: a side stream and two events per device, created on first use
// (make the first call outside a stream capture) and kept for the process.
// The host enqueues one factorisation at a time per device (mu), so that each
// wait binds to its own factorisation's event record.
struct LookaheadCtx {
    std::mutex mu;
    cudaStream_t side;
    cudaEvent_t next_ready;  // main stream: the next block column's updates are in D
    cudaEvent_t diag_done;   // side stream: the next diagonal block is factored and inverted
    int sms;
};

static int lookahead_ctx(LookaheadCtx **out) {
    static std::mutex mu;
    static LookaheadCtx *ctx[64] = {};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(mu);
    if (!ctx[dev]) {
        LookaheadCtx *c = new LookaheadCtx();
        if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->next_ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->diag_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            delete c;
            return GP_ERR_CUDA;
        }
        ctx[dev] = c;
    }
    *out = ctx[dev];
    return GP_OK;
}

// SMs left to the diagonal-block work while the rest of a trailing update
// runs: a fixed share while that update is large, more once it is small and
// the diagonal block would otherwise be the critical path (GP_LOOKAHEAD_SMS
// in the environment overrides the large-update share).
static int lookahead_sms(int64_t m1) {
    static int base = -1;
    if (base < 0) {
        const char *e = getenv("GP_LOOKAHEAD_SMS");
        const int v = e ? atoi(e) : 0;
        base = (v > 0 && v < 128) ? v : 4;
    }
    if (m1 < 8192) return base * 4;
    if (m1 < 16384) return base * 2;
    return base;
}

// Pending updates of rows [r0, r1) of block column k0 (width nb) into A.
static int fold_rows(double *A, int64_t ld, int64_t np, int64_t k0, int64_t nb, int64_t r0,
                     int64_t r1, const MixedWs &w, int64_t *info, cudaStream_t s) {
    const int64_t rows = r1 - r0;
    if (rows <= 0) return GP_OK;
    dim3 g((unsigned)ceil_div(rows, 256 * 4) + 1, (unsigned)nb);
    const int ev = prof_start(s);
    // rows are counted from the block's first column: an offset r0 - k0 shifts the
    // kernel's lower-triangle start (row >= column) accordingly
    fold_delta2_kernel<<<g, 256, 0, s>>>(A + r0 + k0 * ld, ld, w.D + r0 + k0 * np, np, rows, nb,
                                         r0 - k0, info);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_FOLD, 0.0, 16.0 * (double)rows * nb);
    return GP_OK;
}

// Block column k0 (width nb): fold the pending updates of its rows below
// fold_end (k0 > 0; the rest is folded by the caller), factor the diagonal
// block, and, when `inverse`, form W = L_kk^{-1}.
static int diag_block(double *A, int64_t ld, int64_t np, int64_t k0, int64_t nb, int S,
                      const MixedWs &w, double *W, bool inverse, int64_t *info, cudaStream_t s,
                      int64_t fold_end = -1) {
    double *Akk = A + k0 + k0 * ld;
    if (k0 > 0) GP_TRY(fold_rows(A, ld, np, k0, nb, k0, fold_end < 0 ? np : fold_end, w, info, s));
    int ev = prof_start(s);
    GP_TRY(chol_fp64_tiled(Akk, ld, nb, k0, info, s, S == 3));
    prof_stop(ev, s, GP_PROF_DIAG, (double)nb * nb * nb / 3.0, 0.0);
    if (!inverse) return GP_OK;
    ev = prof_start(s);
    GP_TRY(trtri_fp64_blocked(Akk, ld, nb, W, nb, w.tmp, info, s));
    prof_stop(ev, s, GP_PROF_DIAGINV, (double)nb * nb * nb / 3.0, 0.0);
    return GP_OK;
}

// Panel solve L_ik = A_ik L_kk^{-T} of block column k0 (width nb) in place in
// P (m x nb, ld), by tensor-core contractions with the diagonal block's
// inverse W (ld nb).  Blocks wider than 512 are solved in two 512-column
// steps, each with the inverse of its own 512 diagonal sub-block (W's
// diagonal sub-blocks): L_i1 = A_i1 W_11^T, then
// L_i2 = (A_i2 - L_i1 L_21^T) W_22^T; the error of an explicit-inverse solve
// grows with the condition of the block it inverts, and the 512 sub-blocks
// keep it at the 512-block level.  On return w.SA holds the slices of the
// solved panel over the whole width (row bounds per kch columns).
static int panel_solve(double *P, int64_t ld, int64_t m, int64_t nb, const double *Akk,
                       const double *W, int S, const MixedWs &w, int64_t kch, int64_t *info,
                       cudaStream_t s) {
    int *exA = S == 3 ? w.exA : nullptr, *exB = S == 3 ? w.exB : nullptr;
    const int64_t NB = NB_MAX;
    const int64_t h = nb > TC_CHUNK_K ? TC_CHUNK_K : nb;  // first step's width
    const int64_t k5 = TC_CHUNK_K;                         // row bounds of the steps
    TcOperand opA{w.SA, np_of(w), NB, S, 0, 0, exA, tc_ex_ld(NB, k5), k5};
    TcOperand opW{w.SB, NB, NB, S, 0, 0, exB, tc_ex_ld(NB, k5), k5};
    // L_i1 = A_i1 W_11^T
    GP_TRY(split_rows(W, nb, h, h, h, 0, 0, 1, S, w.SB, exB, NB, NB, 0, 0, s, k5));
    GP_TRY(split_rows(P, ld, m, h, h, 0, 0, 0, S, w.SA, exA, np_of(w), NB, 0, 0, s, k5));
    TcOut o1{P, ld, 0, 1.0, 0.0, 0, 0};
    GP_TRY(tc_gemm(opA, opW, m, h, h, o1, 0, 0, info, s));
    if (nb > h) {
        const int64_t h2 = nb - h;
        double *P2 = P + h * ld;
        // A_i2 -= L_i1 L_21^T
        GP_TRY(split_rows(P, ld, m, h, h, 0, 0, 0, S, w.SA, exA, np_of(w), NB, 0, 0, s, k5));
        GP_TRY(split_rows(Akk + h, ld, h2, h, h, 0, 0, 0, S, w.SB, exB, NB, NB, 0, 0, s, k5));
        TcOut o2{P2, ld, 0, -1.0, 1.0, 0, 0};
        GP_TRY(tc_gemm(opA, opW, m, h2, h, o2, 0, 0, info, s));
        // L_i2 = A_i2 W_22^T
        GP_TRY(split_rows(W + h + h * nb, nb, h2, h2, h2, 0, 0, 1, S, w.SB, exB, NB, NB, 0, 0, s,
                          k5));
        GP_TRY(split_rows(P2, ld, m, h2, h2, 0, 0, 0, S, w.SA, exA, np_of(w), NB, 0, 0, s, k5));
        TcOut o3{P2, ld, 0, 1.0, 0.0, 0, 0};
        GP_TRY(tc_gemm(opA, opW, m, h2, h2, o3, 0, 0, info, s));
    }
    // the solved panel, for the trailing update
    return split_rows(P, ld, m, nb, nb, 0, 0, 0, S, w.SA, exA, np_of(w), NB, 0, 0, s, kch);
}

// Without lookahead: every step on the caller's stream, in order.
static int chol_mixed_plain(double *A, int64_t ld, int64_t np, int S, const MixedWs &w,
                            double *winv, int64_t *info, cudaStream_t s) {
    const int64_t NB = chol_block_cols(S), kch = TC_CHUNK_K;
    if (cudaMemsetAsync(w.D, 0, sizeof(float2) * (size_t)np * (size_t)np, s) != cudaSuccess)
        return GP_ERR_CUDA;
    for (int64_t k0 = 0; k0 < np; k0 += NB) {
        const int64_t nb = (np - k0) < NB ? (np - k0) : NB;
        const int64_t m = np - k0 - nb;
        double *W = winv ? winv + (k0 / NB) * NB * NB : w.W;
        GP_TRY(diag_block(A, ld, np, k0, nb, S, w, W, m > 0 || winv, info, s));
        if (m <= 0) break;
        double *Akk = A + k0 + k0 * ld;
        double *P = Akk + nb;
        int *exA = S == 3 ? w.exA : nullptr;
        GP_TRY(panel_solve(P, ld, m, nb, Akk, W, S, w, kch, info, s));
        TcOperand opA{w.SA, np, NB_MAX, S, 0, 0, exA, tc_ex_ld(NB_MAX, kch), kch};
        TcOut o2{w.D + (k0 + nb) + (k0 + nb) * np, np, 2, -1.0, 0.0, 1, 0};
        GP_TRY(tc_gemm(opA, opA, m, m, nb, o2, 0, 0, info, s));
    }
    return GP_OK;
}

int chol_mixed(double *A, int64_t ld, int64_t np, int S, void *ws, double *winv, int64_t *info,
               cudaStream_t s, bool lookahead) {
    MixedWs w = mixed_layout(ws, np, S);
    const int64_t NB = chol_block_cols(S), kch = TC_CHUNK_K;
    ProfContractRole role(GP_PROF_CONTRACT_CHOL);
    if (!lookahead) return chol_mixed_plain(A, ld, np, S, w, winv, info, s);
    LookaheadCtx *la = nullptr;
    GP_TRY(lookahead_ctx(&la));
    std::lock_guard<std::mutex> enqueue(la->mu);
    if (cudaMemsetAsync(w.D, 0, sizeof(float2) * (size_t)np * (size_t)np, s) !=
        cudaSuccess)
        return GP_ERR_CUDA;
    // W = L_kk^{-1} (kept for the gradient's inverse when asked: then the
    // last block's inverse is formed too)
    auto W_of = [&](int64_t k0) { return winv ? winv + (k0 / NB) * NB * NB : w.W; };
    {
        const int64_t nb0 = np < NB ? np : NB;
        GP_TRY(diag_block(A, ld, np, 0, nb0, S, w, W_of(0), np > nb0 || winv, info, s));
    }
    for (int64_t k0 = 0; k0 < np; k0 += NB) {
        const int64_t nb = (np - k0) < NB ? (np - k0) : NB;
        double *Akk = A + k0 + k0 * ld;
        const int64_t m = np - k0 - nb;
        if (m <= 0) break;
        double *P = Akk + nb;  // m x nb panel below the diagonal block
        int *exA = S == 3 ? w.exA : nullptr;
        // L_ik = A_ik L_kk^{-T} (FP64 out), then its slices for the update
        GP_TRY(panel_solve(P, ld, m, nb, Akk, W_of(k0), S, w, kch, info, s));
        TcOperand opA{w.SA, np, NB_MAX, S, 0, 0, exA, tc_ex_ld(NB_MAX, kch), kch};
        // D_22 -= L_ik L_ik^T (lower, double-float), the next block column
        // first: its diagonal block is then folded, factored and inverted on
        // the side stream while the rest of the update runs on the other SMs
        const int64_t k1 = k0 + nb, nbn = m < NB ? m : NB, m1 = m - nbn;
        TcOut o2a{w.D + k1 + k1 * np, np, 2, -1.0, 0.0, 1, 0};
        GP_TRY(tc_gemm(opA, opA, m, nbn, nb, o2a, 0, 0, info, s));
        if (cudaEventRecord(la->next_ready, s) != cudaSuccess ||
            cudaStreamWaitEvent(la->side, la->next_ready, 0) != cudaSuccess)
            return GP_ERR_CUDA;
        GP_TRY(diag_block(A, ld, np, k1, nbn, S, w, W_of(k1), m1 > 0 || winv, info, la->side,
                          k1 + nbn));
        if (cudaEventRecord(la->diag_done, la->side) != cudaSuccess) return GP_ERR_CUDA;
        // the rows below the next diagonal block: folded here on all SMs (a
        // pass over memory), not on the few the side stream gets
        GP_TRY(fold_rows(A, ld, np, k1, nbn, k1 + nbn, np, w, info, s));
        if (m1 > 0) {
            TcOperand opR = opA;
            opR.row_off = nbn;
            TcOut o2b{w.D + (k1 + nbn) + (k1 + nbn) * np, np, 2, -1.0, 0.0, 1, 0};
            const int keep = lookahead_sms(m1);
            o2b.max_ctas = la->sms > 2 * keep ? la->sms - keep : 0;
            GP_TRY(tc_gemm(opR, opR, m1, m1, nb, o2b, 0, 0, info, s));
        }
        if (cudaStreamWaitEvent(s, la->diag_done, 0) != cudaSuccess) return GP_ERR_CUDA;
    }
    return GP_OK;
}

// ---------------------------------------------------------------------------
// Standalone trailing update C (m x m, lower, FP64) -= P P^T, P m x k.
// ---------------------------------------------------------------------------
size_t syrk_ws_bytes(int64_t m, int64_t k, int precision, int S) {
    if (precision == GP_FP64) return 0;
    const int64_t kp = round_up(k, 64);
    return align256(2ull * S * (size_t)m * (size_t)kp) +
           align256(sizeof(int) * (size_t)m * tc_ex_ld(kp));
}

int syrk_lower(double *C, int64_t ldc, const double *P, int64_t ldp, int64_t m, int64_t k,
               int precision, int S, void *ws, int64_t *info, cudaStream_t s) {
    if (precision == GP_FP64)
        return gemm_f64(m, m, k, -1.0, P, ldp, 0, P, ldp, 1, 1.0, C, ldc, 1, info, s);
    const int64_t kp = round_up(k, 64);
    uint16_t *SA = static_cast<uint16_t *>(ws);
    int *ex = S == 3 ? reinterpret_cast<int *>(static_cast<char *>(ws) +
                                               align256(2ull * S * (size_t)m * (size_t)kp))
                     : nullptr;
    GP_TRY(split_rows(P, ldp, m, kp, k, 0, 0, 0, S, SA, ex, m, kp, 0, 0, s));
    // one contraction per 512-deep chunk, accumulated in FP64
    for (int64_t k0 = 0; k0 < kp; k0 += TC_CHUNK_K) {
        const int64_t kc = (kp - k0) < TC_CHUNK_K ? (kp - k0) : TC_CHUNK_K;
        TcOperand op{SA, m, kp, S, 0, k0, ex, tc_ex_ld(kp)};
        TcOut o{C, ldc, 0, -1.0, 1.0, 1, 0};
        GP_TRY(tc_gemm(op, op, m, m, kc, o, 0, 0, info, s));
    }
    return GP_OK;
}

}  // namespace gp
