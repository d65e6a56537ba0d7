// tc_gemm.cu -- the dense contractions of the blocked Cholesky (Sec. 2.1:
// "most of the total work is in the matrix multiplications") and of the
// gradient's inverse, on the sm_103a tensor cores, with FP64 operands
// carried as 16-bit slices.
//
// Operand splitting (row-scaled).  For operand row r let 2^e_r bound its
// entries over a 512-deep chunk of K.
//   Mixed form (three FP16 slices, "normalized"): with y = x 2^{7-e_r},
//   s0 = round(y), an integer in [-128, 128]; s1 = fp16(y - s0);
//   s2 = fp16(y - s0 - s1), so y is carried to about 2^-25.  The slice
//   products s_p t_q with p + q < 3 are kept (the dropped ones are below
//   2^-28 of the row maxima); the epilogue scales each chunk's sums by
//   2^{e_a + e_b - 14}.
//   FP64-grade form (five BF16 slices, "scaled"): every slice is an integer
//   q_p in [-128, 128] times 2^{e_r-7-8p}, carrying x to 2^-40 of the row
//   bound; the 15 products with p + q < 5 are kept.
// The products of one group d = p + q share their scale for a given output
// (r, c); group 0 (integer products) is exact in an FP32 accumulator for
// K <= 1024, and in the integer form groups 1 and 2 are too for K <= 512.
// Groups get their own TMEM accumulators: the mixed form one per group (hi,
// d1, d2), the FP64-grade form groups 0, 1, 2 and a fourth for groups 3 and
// 4.  The epilogue adds them in FP64 or in double-float.
//
// Two kernels, both persistent (one CTA per SM walks a static tile schedule
// of 128 x 128 output tiles, grouped 16 tile-rows at a time so the operand
// tiles in flight stay in L2):
//   tc_gemm_kernel<NACC> (five slices): 10 warps.
//     warp 0     TMA producer (one thread): a 6-stage ring of 32 KB stages
//                (one slice pair: A and B 128 x 64 boxes, 128-byte swizzle).
//     warp 1     TMEM owner (512 columns: 2 tile buffers x 2 accumulators, or
//                one buffer x 4) and MMA issuer (one thread):
//                tcgen05.mma.cta_group::1.kind::f16, 128 x 128 x 16 per
//                instruction; tcgen05.commit frees stages and hands finished
//                accumulators to the epilogue.
//     warps 2-9  epilogue, two warps per TMEM lane quarter (32 rows x 64
//                columns each): tcgen05.ld of the accumulators, output in
//                FP64 (C = beta C + alpha acc) or as a double-float FP32 pair
//                (C += alpha acc, error-free sums), one row per thread so that
//                every warp access covers 32 consecutive rows of one column.
//                The previous output values are read one 8-column step ahead.
//   tc_gemm3_kernel (three slices): stages that carry every slice, two MMA
//   issuers and an epilogue staged through registers (described with it).
// Every mbarrier wait is bounded (1 s); a wait that gives up sets
// *info = -1, the roles wind down (the producer waits, bounded, for its
// copies in flight) and TMEM is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "internal.h"
#include "kern_df.cuh"
#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace gp {

constexpr int TC_BM = 128;
constexpr int TC_BN = 128;
constexpr int TC_BK = 64;
constexpr int TC_STAGES = 6;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 /*barriers*/ + 1024 /*align*/;
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr int TC_GROUP = 16;  // tile rows per scheduling group
constexpr int TC_MAX_PAIRS = 15;
constexpr int TC_EPI_WARPS = 8;                     // two per TMEM lane quarter
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);  // producer, MMA, epilogue

struct TcGemmArgs {
    void *C;
    int64_t ldc;
    int out_mode;  // 0: FP64 C = beta C + alpha v;
                   // 2: FP32 pair (hi, lo) C += alpha v in double-float
    double alpha, beta;
    int lower;
    int64_t diag_off;
    int64_t M, N;
    int a_row_off, b_row_off, a_k_off, b_k_off;
    int kblocks;
    int tri_k;
    int64_t tri_off;
    int kchunk;  // > 0: flush the accumulators every kchunk K-blocks (one epilogue
                 // pass per chunk, out_mode 2 accumulates the chunks in double-float)
    int tiles_m, tiles_n;
    int npairs;
    int pa[TC_MAX_PAIRS], pb[TC_MAX_PAIRS];
    int acc_of[TC_MAX_PAIRS];    // TMEM accumulator of each slice pair
    int first_of[TC_MAX_PAIRS];  // pair opens its accumulator
    int nacc, nbuf;              // accumulators per tile, tile buffers (nacc*nbuf <= 4)
    uint32_t idesc;              // MMA instruction descriptor (FP16 or BF16 operands)
    const int *ex_a, *ex_b;      // normalized slices: row exponents per kch-chunk, else null
    int64_t ex_ld_a, ex_ld_b;
    int kch;                     // K width of one row bound (and of one flush of a deep contraction)
    int64_t *info;
    // three-slice kernel, chunked contraction into an FP64 output: C above is
    // the double-float running sum (written, not read, by a tile's first
    // chunk); the last chunk writes Cf = alpha_f64 (running sum + chunk)
    // instead (a tile with no K range writes zeros)
    int fuse_f64;
    double *Cf;
    int64_t ldcf;
    double alpha_f64;
};

struct TileInfo {
    int tm, tn, kb_lo, kb_hi;
    bool skip;
};

// Accumulation units of a tile: one (the whole K range, even if empty) when
// kchunk == 0, else the non-empty kchunk-aligned pieces of [kb_lo, kb_hi).
__device__ __forceinline__ int tile_chunks(const TcGemmArgs &a, int kb_lo, int kb_hi) {
    if (a.kchunk <= 0) return 1;
    if (kb_lo >= kb_hi) return a.fuse_f64 ? 1 : 0;
    return (kb_hi - 1) / a.kchunk - kb_lo / a.kchunk + 1;
}

__device__ __forceinline__ void chunk_range(const TcGemmArgs &a, int kb_lo, int kb_hi, int c,
                                            int &lo, int &hi) {
    if (a.kchunk <= 0) {
        lo = kb_lo;
        hi = kb_hi;
        return;
    }
    const int c0 = kb_lo / a.kchunk + c;
    lo = max(kb_lo, c0 * a.kchunk);
    hi = min(kb_hi, (c0 + 1) * a.kchunk);
}

__device__ __forceinline__ TileInfo tile_at(const TcGemmArgs &a, int t) {
    TileInfo ti;
    const int per_group = TC_GROUP * a.tiles_n;
    const int g = t / per_group;
    const int rem = t - g * per_group;
    const int rows_in_group = min(TC_GROUP, a.tiles_m - g * TC_GROUP);
    ti.tn = rem / rows_in_group;
    ti.tm = g * TC_GROUP + rem % rows_in_group;
    const int64_t row0 = (int64_t)ti.tm * TC_BM, col0 = (int64_t)ti.tn * TC_BN;
    ti.skip = a.lower && (col0 > row0 + (TC_BM - 1) + a.diag_off);
    ti.kb_lo = 0;
    if (a.tri_k) {
        int64_t k0 = col0 - a.tri_off;
        ti.kb_lo = k0 > 0 ? (int)(k0 / TC_BK) : 0;
    }
    ti.kb_hi = a.kblocks;
    return ti;
}

// Error-free transformations in FP32 (never contracted into FMAs).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

constexpr int TC_EG = 8;  // columns per epilogue step (two steps' loads in flight)

// Previous output values (FP64 or an FP32 pair: 8 bytes either way) of one
// row and TC_EG columns; masked entries read as 0.
__device__ __forceinline__ void fetch_old(const TcGemmArgs &a, bool need_old, int64_t row,
                                          bool row_ok, int64_t colb,
                                          unsigned long long (&o)[TC_EG]) {
    const unsigned long long *src =
        static_cast<const unsigned long long *>(a.C) + row + colb * a.ldc;
#pragma unroll
    for (int j = 0; j < TC_EG; ++j) {
        const int64_t col = colb + j;
        const bool ok = need_old && row_ok && col < a.N && (!a.lower || row + a.diag_off >= col);
        o[j] = ok ? src[j * a.ldc] : 0ull;
    }
}

// One TC_EG-column step of an epilogue warp: accumulators from TMEM (column
// tcol of the first one), previous values in old[], result written to C.
template <int NACC>
__device__ __forceinline__ void epilogue_group(const TcGemmArgs &args, uint32_t tcol, bool has_acc,
                                               int64_t row, bool row_ok, int64_t colb,
                                               float alpha_f, int ea, int ebr, int lane0,
                                               const unsigned long long (&old)[TC_EG]) {
    constexpr int nacc = NACC;
    // normalized slices: this chunk's sums carry the factor 2^{e_a + e_b - 14};
    // lane lane0 + j holds e_b of column j in ebr (a tile with no K range has
    // zero sums and reads no exponents)
    int ksc[TC_EG];
#pragma unroll
    for (int j = 0; j < TC_EG; ++j) {
        const int eb = __shfl_sync(0xffffffffu, ebr, lane0 + j);
        ksc[j] = (args.ex_b && has_acc) ? max(-252, min(ea + eb - 14, 252)) : 0;
    }
    uint32_t a0[TC_EG], a1[TC_EG], a2[TC_EG], a3[TC_EG];
#pragma unroll
    for (int j = 0; j < TC_EG; ++j) a0[j] = a1[j] = a2[j] = a3[j] = 0u;
    if (has_acc) {
        tmem_ld_32x32b_x8(tcol, a0);
        tmem_ld_32x32b_x8(tcol + TC_BN, a1);
        if (nacc > 2) tmem_ld_32x32b_x8(tcol + 2 * TC_BN, a2);
        if (nacc > 3) tmem_ld_32x32b_x8(tcol + 3 * TC_BN, a3);
        tmem_ld_wait();
    }
    bool okc[TC_EG];
#pragma unroll
    for (int j = 0; j < TC_EG; ++j) {
        const int64_t col = colb + j;
        okc[j] = row_ok && col < args.N && (!args.lower || row + args.diag_off >= col);
    }
    if (args.out_mode == 2) {
        // double-float: v = a0 + a1 + a2 + a3 as an unevaluated pair (h, l),
        // then C (hi, lo) += alpha v, all in FP32
        float2 *dst = static_cast<float2 *>(args.C) + row + colb * args.ldc;
#pragma unroll
        for (int j = 0; j < TC_EG; ++j) {
            const float ox = __uint_as_float(static_cast<uint32_t>(old[j]));
            const float oy = __uint_as_float(static_cast<uint32_t>(old[j] >> 32));
            float h, l;
            two_sum(__uint_as_float(a0[j]), __uint_as_float(a1[j]), h, l);
            if (nacc > 2) {
                float m, e, l2, e2;
                two_sum(__uint_as_float(a2[j]), __uint_as_float(a3[j]), m, e);
                two_sum(l, m, l2, e2);
                two_sum(h, l2, h, l);
                l = __fadd_rn(l, __fadd_rn(e2, e));
            }
            // alpha 2^k in two exact power-of-two factors (|k| <= 252 fits)
            const int k1 = ksc[j] / 2, k2 = ksc[j] - k1;
            const float f1 = __fmul_rn(alpha_f, __int_as_float((k1 + 127) << 23));
            const float f2 = __int_as_float((k2 + 127) << 23);
            h = __fmul_rn(__fmul_rn(h, f1), f2);
            l = __fmul_rn(__fmul_rn(l, f1), f2);
            float s1, e1, hi, lo;
            two_sum(ox, h, s1, e1);
            e1 = __fadd_rn(e1, __fadd_rn(oy, l));
            two_sum(s1, e1, hi, lo);
            if (okc[j]) dst[j * args.ldc] = make_float2(hi, lo);
        }
    } else {
        double *dst = static_cast<double *>(args.C) + row + colb * args.ldc;
#pragma unroll
        for (int j = 0; j < TC_EG; ++j) {
            // conversions and the exact 2^k scaling by integer operations
            // (sums of FP32 values are zero or at least 2^-149 in magnitude,
            // so the scaled value stays a normal FP64 number)
            double v = f32_to_f64(__uint_as_float(a0[j])) + f32_to_f64(__uint_as_float(a1[j]));
            if (nacc > 2)
                v += f32_to_f64(__uint_as_float(a2[j])) + f32_to_f64(__uint_as_float(a3[j]));
            {
                const long long b = __double_as_longlong(v);
                if (b & 0x7FFFFFFFFFFFFFFFll)
                    v = __longlong_as_double(b + (static_cast<long long>(ksc[j]) << 52));
            }
            if (args.beta != 0.0)
                v = fma(args.beta, __longlong_as_double(static_cast<long long>(old[j])),
                        args.alpha * v);
            else if (args.alpha == -1.0)
                v = -v;
            else if (args.alpha != 1.0)
                v = args.alpha * v;
            if (okc[j]) dst[j * args.ldc] = v;
        }
    }
}

template <int NACC>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   TcGemmArgs args) {
    extern __shared__ uint8_t smem_raw[];
    if (args.info && failed(args.info)) return;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *tfull = empty + TC_STAGES;   // [2] accumulator ready
    uint64_t *tempty = tfull + 2;          // [2] accumulator drained
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], TC_EPI_WARPS);
        }
        mbar_init(drain, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TC_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int ntiles = args.tiles_m * args.tiles_n;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        uint32_t it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const int ra = ti.tm * TC_BM + args.a_row_off, rb = ti.tn * TC_BN + args.b_row_off;
            const int nch = tile_chunks(args, ti.kb_lo, ti.kb_hi);
            for (int c = 0; c < nch && ok; ++c) {
            int clo, chi;
            chunk_range(args, ti.kb_lo, ti.kb_hi, c, clo, chi);
            for (int p = 0; p < args.npairs && ok; ++p) {
                for (int kb = clo; kb < chi; ++kb, ++it) {
                    const uint32_t s = it % TC_STAGES, use = it / TC_STAGES;
                    if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    if (abort_flag) {
                        ok = false;
                        break;
                    }
                    uint8_t *a_s = smem + s * TC_STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[s], TC_STAGE_BYTES);
                    const int kx = kb * TC_BK;
                    tma_load_3d(a_s, &tmA, &full[s], args.a_k_off + kx, ra, args.pa[p]);
                    tma_load_3d(a_s + TC_A_BYTES, &tmB, &full[s], args.b_k_off + kx, rb, args.pb[p]);
                }
            }
            }
        }
        if (!ok) abort_flag = 1;
        // drain: copies still in flight must land before the CTA exits
        for (uint32_t j = (it > TC_STAGES ? it - TC_STAGES : 0); j < it; ++j)
            mbar_wait(&full[j % TC_STAGES], (j / TC_STAGES) & 1);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = args.idesc;
        uint32_t it = 0, local = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const int nch = tile_chunks(args, ti.kb_lo, ti.kb_hi);
            for (int c = 0; c < nch && ok; ++c) {
            int clo, chi;
            chunk_range(args, ti.kb_lo, ti.kb_hi, c, clo, chi);
            const uint32_t buf = local % args.nbuf, u = local / args.nbuf;
            if (u > 0 && !mbar_wait(&tempty[buf], (u - 1) & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            for (int p = 0; p < args.npairs && ok; ++p) {
                const uint32_t acc = tmem + (buf * args.nacc + args.acc_of[p]) * TC_BN;
                const bool first_of_acc = args.first_of[p] != 0;
                for (int kb = clo; kb < chi; ++kb, ++it) {
                    const uint32_t s = it % TC_STAGES, use = it / TC_STAGES;
                    if (!mbar_wait(&full[s], use & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(smem + s * TC_STAGE_BYTES);
                    const uint32_t b_addr = a_addr + TC_A_BYTES;
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k) {
                        const uint32_t accumulate = (first_of_acc && kb == clo && k == 0) ? 0u : 1u;
                        mma_f16_ss(acc, sdesc_sw128(a_addr + k * 32), sdesc_sw128(b_addr + k * 32),
                                   idesc, accumulate);
                    }
                    mma_commit(&empty[s]);
                }
            }
            mma_commit(&tfull[buf]);
            ++local;
            }
        }
        if (!ok) abort_flag = 1;
        mma_commit(drain);
        mbar_wait(drain, 0);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        // warps 2-9: TMEM lane quarter q = warp % 4 (the quarter a warp may
        // access), column half h; each warp owns 32 rows x 64 columns
        const int q = warp & 3;
        const int cbeg = ((warp - 2) >> 2) * (TC_BN / 2);
        uint32_t local = 0;
        const float alpha_f = static_cast<float>(args.alpha);
        const bool need_old = args.out_mode == 2 || args.beta != 0.0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const int nch = tile_chunks(args, ti.kb_lo, ti.kb_hi);
            bool stop = false;
            const int64_t row = (int64_t)ti.tm * TC_BM + q * 32 + lane;
            const bool row_ok = row < args.M;
            const int64_t col0 = (int64_t)ti.tn * TC_BN + cbeg;
            for (int c = 0; c < nch; ++c) {
            int clo, chi;
            chunk_range(args, ti.kb_lo, ti.kb_hi, c, clo, chi);
            const uint32_t buf = local % args.nbuf, u = local / args.nbuf;
            unsigned long long cur[TC_EG], nxt[TC_EG];
            fetch_old(args, need_old, row, row_ok, col0, cur);  // in flight during the MMAs
            // row exponents of this flush's 512-deep chunk (normalized slices):
            // this thread's A row, and the B rows of columns col0 + lane and
            // col0 + 32 + lane, shuffled to the column steps below
            int ea = 0, eb0 = 0, eb1 = 0;
            if (args.ex_b && clo < chi) {
                const int64_t cha = (args.a_k_off + (int64_t)clo * TC_BK) / args.kch;
                const int64_t chb = (args.b_k_off + (int64_t)clo * TC_BK) / args.kch;
                if (row_ok) ea = args.ex_a[(args.a_row_off + row) * args.ex_ld_a + cha];
                const int64_t c0 = col0 + lane, c1 = col0 + 32 + lane;
                if (c0 < args.N) eb0 = args.ex_b[(args.b_row_off + c0) * args.ex_ld_b + chb];
                if (c1 < args.N) eb1 = args.ex_b[(args.b_row_off + c1) * args.ex_ld_b + chb];
            }
            bool ok = mbar_wait(&tfull[buf], u & 1);
            ok = __all_sync(0xffffffffu, ok) && !abort_flag;
            if (!ok) {
                if (lane == 0) abort_flag = 1;
                stop = true;
                break;
            }
            tc_fence_after();
            const bool has_acc = clo < chi;
            const uint32_t tmem_col = tmem + (static_cast<uint32_t>(q * 32) << 16) + cbeg +
                                      buf * args.nacc * TC_BN;
            // two named buffers, so that every array index is static
            for (int g = 0; g < TC_BN / 2; g += 2 * TC_EG) {
                fetch_old(args, need_old, row, row_ok, col0 + g + TC_EG, nxt);
                const int ebr = g < 32 ? eb0 : eb1;
                epilogue_group<NACC>(args, tmem_col + g, has_acc, row, row_ok, col0 + g, alpha_f,
                                     ea, ebr, g & 31, cur);
                if (g + 2 * TC_EG < TC_BN / 2)
                    fetch_old(args, need_old, row, row_ok, col0 + g + 2 * TC_EG, cur);
                epilogue_group<NACC>(args, tmem_col + g + TC_EG, has_acc, row, row_ok,
                                     col0 + g + TC_EG, alpha_f, ea, ebr, (g + TC_EG) & 31, nxt);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            ++local;
            }
            if (stop) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0 && args.info) set_info(args.info, -1);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}


// ---------------------------------------------------------------------------
// Three-slice (mixed form) kernel: one TMEM accumulator per product group
// d = p + q (hi: d = 0, d1, d2), two MMA issuers, epilogue through registers.
//
// A stage carries every slice of both operands for one 64-deep K block (two
// 3-D boxes of 3 x 128 x 64 FP16, 96 KB), so each fetched byte feeds all the
// products that use it (4 KB of operands per 128 x 128 x 16 instruction
// instead of 8 KB).  Issuer A (warp 1) forms (0,0) into hi and (0,1), (1,0)
// into d1; issuer B (warp 2) forms (0,2), (1,1), (2,0) into d2: three
// instructions per stage and k-step each, issued concurrently (one issuing
// thread sustains about one instruction per 150 cycles, two together about
// one per 88).  TMEM: hi [0, 128), d1 [128, 256), d2 [256, 384); columns
// [384, 512) hold the epilogue's staged high parts.
//
// Epilogue (EPI warps from warp 3 on, EPI / 4 per TMEM lane quarter, each
// 32 rows x 512 / EPI columns): as soon as a unit's accumulators are
// complete it reads hi and d1, adds them error-free into a double-float pair
// (h, l) per entry, writes h to the staging columns, keeps l in registers
// and frees hi and d1 for issuer A; then it adds d2 into l and frees d2 for
// issuer B.  The read-modify-write of the outputs then runs while the next
// unit's instructions execute; its old values are prefetched into L2 while
// the unit's own instructions execute.  That output pass is latency bound
// (dependent FP32 chains, old-value loads): where every tile is a single
// 512-deep unit (the Cholesky's trailing updates, one unit per output) it
// outlasts the unit's instructions with 8 warps, and 16 warps (two steps of
// old values in flight each, to stay within the register budget) take it
// about a quarter faster; deep contractions, whose units are several
// instructions long per output, keep 8 warps, which leave the issuers more
// of the SM.
// ---------------------------------------------------------------------------
constexpr int T3_STAGES = 2;
constexpr int T3_SLICE = TC_BM * TC_BK * 2;  // 16 KB: one slice of one operand
constexpr int T3_OPER = 3 * T3_SLICE;        // 48 KB: every slice of one operand
constexpr int T3_STAGE = 2 * T3_OPER;        // 96 KB
constexpr int T3_SMEM = T3_STAGES * T3_STAGE + 1024 /*barriers*/ + 1024 /*align*/;
constexpr int T3_EG = 4;  // columns per output step

// Epilogue shape for EPI epilogue warps (8 or 16).
template <int EPI>
struct T3Epi {
    static constexpr int THREADS = 32 * (3 + EPI);  // producer, two issuers, epilogue
    static constexpr int COLS = TC_BN * 4 / EPI;    // columns per epilogue warp
    static constexpr int NEB = COLS / 32;           // B-row exponents per lane
    static constexpr int INFL = EPI >= 16 ? 2 : 4;  // output steps with old values in flight
    static_assert(EPI == 8 || EPI == 16, "8 or 16 epilogue warps");
};

// Previous output values of T3_EG consecutive columns of this thread's row:
// p points at column cl of the row (8-byte entries, stride ld8 bytes), lim is
// the row's first column (local) that is not written; masked entries read 0.
__device__ __forceinline__ void t3_fetch(const char *p, int64_t ld8, int cl, int lim,
                                         unsigned long long (&o)[T3_EG]) {
#pragma unroll
    for (int j = 0; j < T3_EG; ++j)
        o[j] = cl + j < lim ? *reinterpret_cast<const unsigned long long *>(p + j * ld8) : 0ull;
}

// One output step: columns cl + j of this thread's row from the pairs
// (h[j], l[j]) (the unit's unscaled sums), old values in old[].  The sums
// carry the factor alpha 2^{e_a + e_b - 14}: fa = alpha 2^{e_a} is this
// row's, e_b of column cl + j sits in lane lane0 + j of ebr.  Row exponents
// lie in [-100, 120] (the packing clamps them), so fa and 2^{e_b - 14} are
// normal and their product is exact wherever the scaled result is
// representable (a power of two down to 2^-149).
__device__ __forceinline__ void t3_store(const TcGemmArgs &args, const float *h_, const float *l_,
                                         char *p, int64_t ld8, int cl, int lim, float fa, int ea,
                                         int ebr, int lane0, const unsigned long long (&old)[T3_EG],
                                         char *pf, int64_t ld8f, bool to_f64) {
#pragma unroll
    for (int j = 0; j < T3_EG; ++j) {
        const int eb = __shfl_sync(0xffffffffu, ebr, lane0 + j);
        if (args.out_mode == 2) {
            const float f = __fmul_rn(fa, __int_as_float((eb + 113) << 23));
            const float ox = __uint_as_float(static_cast<uint32_t>(old[j]));
            const float oy = __uint_as_float(static_cast<uint32_t>(old[j] >> 32));
            const float h = __fmul_rn(h_[j], f), l = __fmul_rn(l_[j], f);
            float s1, e1, hi, lo;
            two_sum(ox, h, s1, e1);
            e1 = __fadd_rn(e1, __fadd_rn(oy, l));
            two_sum(s1, e1, hi, lo);
            if (to_f64) {
                // the last chunk of a fused chunked contraction: FP64 out
                double v = f32_to_f64(hi) + f32_to_f64(lo);
                if (args.alpha_f64 == -1.0) v = -v;
                else if (args.alpha_f64 != 1.0) v *= args.alpha_f64;
                if (cl + j < lim) *reinterpret_cast<double *>(pf + j * ld8f) = v;
            } else if (cl + j < lim) {
                *reinterpret_cast<float2 *>(p + j * ld8) = make_float2(hi, lo);
            }
        } else {
            // (h + l) 2^{e_a + e_b - 14}: the scaling and the conversions by
            // integer operations, one FP64 add (the FP64 pipe runs at 1/64
            // of the FP32 rate); alpha = +-1 by the sign bit
            const int k = ea + eb - 14;
            double v = f32_to_f64_scaled(h_[j], k) + f32_to_f64_scaled(l_[j], k);
            if (args.beta != 0.0)
                v = fma(args.beta, __longlong_as_double(static_cast<long long>(old[j])),
                        args.alpha * v);
            else if (args.alpha == -1.0)
                v = -v;
            else if (args.alpha != 1.0)
                v = args.alpha * v;
            if (cl + j < lim) *reinterpret_cast<double *>(p + j * ld8) = v;
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(T3Epi<EPI>::THREADS, 1)
    tc_gemm3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    TcGemmArgs args) {
    using E = T3Epi<EPI>;
    extern __shared__ uint8_t smem_raw[];
    if (args.info && failed(args.info)) return;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + T3_STAGES * T3_STAGE);
    uint64_t *empty = full + T3_STAGES;  // both issuers' commits
    uint64_t *fullA = empty + T3_STAGES;  // hi, d1 of a unit complete
    uint64_t *fullB = fullA + 1;          // d2 complete
    uint64_t *freeA = fullB + 1;          // hi, d1 read by every epilogue warp
    uint64_t *freeB = freeA + 1;          // d2 read by every epilogue warp
    uint64_t *drain = freeB + 1;          // [2] each issuer's last instructions done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 2);
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < T3_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 2);
        }
        mbar_init(fullA, 1);
        mbar_init(fullB, 1);
        mbar_init(freeA, EPI);
        mbar_init(freeB, EPI);
        mbar_init(&drain[0], 1);
        mbar_init(&drain[1], 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TC_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int ntiles = args.tiles_m * args.tiles_n;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: one stage per K block ----------------
        // operand slices are re-read by other tiles: kept in L2 in preference
        // to the outputs, which each unit reads and writes once
        const uint64_t pol_in = l2_policy_evict_last();
        uint32_t it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const int ra = ti.tm * TC_BM + args.a_row_off, rb = ti.tn * TC_BN + args.b_row_off;
            const int nch = tile_chunks(args, ti.kb_lo, ti.kb_hi);
            for (int c = 0; c < nch && ok; ++c) {
                int clo, chi;
                chunk_range(args, ti.kb_lo, ti.kb_hi, c, clo, chi);
                for (int kb = clo; kb < chi; ++kb, ++it) {
                    const uint32_t s = it % T3_STAGES, use = it / T3_STAGES;
                    if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    if (abort_flag) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = smem + s * T3_STAGE;
                    mbar_arrive_expect_tx(&full[s], T3_STAGE);
                    const int kx = kb * TC_BK;
                    tma_load_3d_hint(st, &tmA, &full[s], args.a_k_off + kx, ra, 0, pol_in);
                    tma_load_3d_hint(st + T3_OPER, &tmB, &full[s], args.b_k_off + kx, rb, 0, pol_in);
                }
            }
        }
        if (!ok) abort_flag = 1;
        for (uint32_t j = (it > T3_STAGES ? it - T3_STAGES : 0); j < it; ++j)
            mbar_wait(&full[j % T3_STAGES], (j / T3_STAGES) & 1);
    } else if ((warp == 1 || warp == 2) && lane == 0) {
        // ---------------- MMA issuers ----------------
        const bool isB = warp == 2;
        const uint32_t idesc = args.idesc;
        uint32_t it = 0, local = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const int nch = tile_chunks(args, ti.kb_lo, ti.kb_hi);
            for (int c = 0; c < nch && ok; ++c) {
                int clo, chi;
                chunk_range(args, ti.kb_lo, ti.kb_hi, c, clo, chi);
                if (local > 0 && !mbar_wait(isB ? freeB : freeA, (local - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc0 = isB ? tmem + 2 * TC_BN : tmem;
                const uint32_t acc1 = isB ? acc0 : tmem + TC_BN;
                // the pair that opens acc0: A (0,0) into hi, B (0,2) into d2
                const int q0 = isB ? 2 : 0;
                for (int kb = clo; kb < chi; ++kb, ++it) {
                    const uint32_t s = it % T3_STAGES, use = it / T3_STAGES;
                    if (!mbar_wait(&full[s], use & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(smem + s * T3_STAGE);
                    const uint32_t b_addr = a_addr + T3_OPER;
                    const uint32_t first = kb == clo ? 0u : 1u;
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)
                        mma_f16_ss(acc0, sdesc_sw128(a_addr + k * 32),
                                   sdesc_sw128(b_addr + q0 * T3_SLICE + k * 32), idesc,
                                   k == 0 ? first : 1u);
                    if (!isB) {
                        // d1: (0,1) opens it, then (1,0)
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_f16_ss(acc1, sdesc_sw128(a_addr + k * 32),
                                       sdesc_sw128(b_addr + T3_SLICE + k * 32), idesc,
                                       k == 0 ? first : 1u);
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_f16_ss(acc1, sdesc_sw128(a_addr + 1 * T3_SLICE + k * 32),
                                       sdesc_sw128(b_addr + 0 * T3_SLICE + k * 32), idesc, 1u);
                    } else {
                        // d2: (0,2) opened it above, then (1,1), (2,0)
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_f16_ss(acc0, sdesc_sw128(a_addr + 1 * T3_SLICE + k * 32),
                                       sdesc_sw128(b_addr + 1 * T3_SLICE + k * 32), idesc, 1u);
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k)
                            mma_f16_ss(acc0, sdesc_sw128(a_addr + 2 * T3_SLICE + k * 32),
                                       sdesc_sw128(b_addr + 0 * T3_SLICE + k * 32), idesc, 1u);
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(isB ? fullB : fullA);
                ++local;
            }
        }
        if (!ok) abort_flag = 1;
        mma_commit(&drain[isB ? 1 : 0]);
        mbar_wait(&drain[isB ? 1 : 0], 0);
    } else if (warp >= 3) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;                        // TMEM lane quarter of this warp
        const int cbeg = ((warp - 3) >> 2) * E::COLS;  // its columns in the tile
        uint32_t local = 0;
        const float alpha_f = static_cast<float>(args.alpha);
        const bool need_old = args.out_mode == 2 || args.beta != 0.0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const int nch = tile_chunks(args, ti.kb_lo, ti.kb_hi);
            bool stop = false;
            const int64_t row = (int64_t)ti.tm * TC_BM + q * 32 + lane;
            const bool row_ok = row < args.M;
            const int64_t col0 = (int64_t)ti.tn * TC_BN + cbeg;
            for (int c = 0; c < nch; ++c) {
                int clo, chi;
                chunk_range(args, ti.kb_lo, ti.kb_hi, c, clo, chi);
                const bool has_acc = clo < chi;
                // this thread's row: its entries at p_row + cl * ld8 (local
                // column cl), written while cl < lim
                int lim = 0;
                if (row_ok) {
                    int64_t e = args.N;
                    if (args.lower && row + args.diag_off + 1 < e) e = row + args.diag_off + 1;
                    e -= col0;
                    lim = e <= 0 ? 0 : (e >= E::COLS ? E::COLS : (int)e);
                }
                const int64_t ld8 = args.ldc * 8;
                char *p_row = static_cast<char *>(args.C) + (row_ok ? (row + col0 * args.ldc) * 8 : 0);
                // fused chunked FP64 output: the first chunk starts the running
                // sum (no old values), the last one writes the FP64 result
                const bool fresh = args.fuse_f64 && c == 0;
                const bool to_f64 = args.fuse_f64 && c == nch - 1;
                const bool read_old = need_old && !fresh;
                const int64_t ld8f = args.ldcf * 8;
                char *pf_row = (to_f64 && row_ok)
                                   ? reinterpret_cast<char *>(args.Cf) + (row + col0 * args.ldcf) * 8
                                   : nullptr;
                // old values of this row into L2 while the unit's instructions
                // run (one line request per column and lane pair)
                if (read_old)
                    for (int j = 0; j < lim; ++j)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(p_row + j * ld8));
                // row exponents of this unit's 512-deep chunk: this thread's A
                // row, and the B rows of columns col0 + 32 m + lane
                // (unscaled sums: ea = 0, eb = 14)
                int ea = 0, eb[E::NEB];
#pragma unroll
                for (int m = 0; m < E::NEB; ++m) eb[m] = 14;
                if (args.ex_b && has_acc) {
                    const int64_t cha = (args.a_k_off + (int64_t)clo * TC_BK) / args.kch;
                    const int64_t chb = (args.b_k_off + (int64_t)clo * TC_BK) / args.kch;
                    if (row_ok) ea = args.ex_a[(args.a_row_off + row) * args.ex_ld_a + cha];
#pragma unroll
                    for (int m = 0; m < E::NEB; ++m) {
                        const int64_t cm = col0 + 32 * m + lane;
                        if (cm < args.N) eb[m] = args.ex_b[(args.b_row_off + cm) * args.ex_ld_b + chb];
                    }
                }
                const int flim = read_old ? lim : 0;  // columns whose old values are read
                const float fa = __fmul_rn(alpha_f, __int_as_float((ea + 127) << 23));
                // a ring of E::INFL output steps of old values; the first ones
                // are in flight during the wait
                unsigned long long old[E::INFL][T3_EG];
#pragma unroll
                for (int g = 0; g < E::INFL - 1; ++g)
                    t3_fetch(p_row + g * T3_EG * ld8, ld8, g * T3_EG, flim, old[g]);
                bool ok = mbar_wait(fullB, local & 1) && mbar_wait(fullA, local & 1);
                ok = __all_sync(0xffffffffu, ok) && !abort_flag;
                if (!ok) {
                    if (lane == 0) abort_flag = 1;
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t tl = tmem + (static_cast<uint32_t>(q * 32) << 16) + cbeg;
                const uint32_t th = tl + 3 * TC_BN;  // staged high parts
                float L[E::COLS];
                if (has_acc) {
#pragma unroll
                    for (int g = 0; g < E::COLS; g += 16) {
                        uint32_t a0[16], a1[16];
                        tmem_ld_32x32b_x16(tl + g, a0);
                        tmem_ld_32x32b_x16(tl + TC_BN + g, a1);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float h;
                            two_sum(__uint_as_float(a0[j]), __uint_as_float(a1[j]), h, L[g + j]);
                            a0[j] = __float_as_uint(h);
                        }
                        // the store reads a0 asynchronously: wait before the
                        // registers are reused
                        tmem_st_32x32b_x16(th + g, a0);
                        tmem_st_wait();
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < E::COLS; ++j) L[j] = 0.0f;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(freeA);
                if (has_acc) {
#pragma unroll
                    for (int g = 0; g < E::COLS; g += 16) {
                        uint32_t a2[16];
                        tmem_ld_32x32b_x16(tl + 2 * TC_BN + g, a2);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) L[g + j] = __fadd_rn(L[g + j], __uint_as_float(a2[j]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(freeB);
                // outputs, 16 columns per block: h from the staging columns,
                // l from L[0..15] (L rotates by 16 per block, so that the loop
                // stays rolled: unrolled over 128 columns the code outgrows the
                // instruction cache); step g's old values were requested
                // E::INFL - 1 steps earlier
                static_assert(16 % T3_EG == 0 && (16 / T3_EG) % E::INFL == 0, "ring");
                constexpr int NSTEP = E::COLS / T3_EG;
#pragma unroll 1
                for (int blk = 0; blk < E::COLS / 16; ++blk) {
                    float H[16];
                    if (has_acc) {
                        uint32_t hv[16];
                        tmem_ld_32x32b_x16(th + blk * 16, hv);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) H[j] = __uint_as_float(hv[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) H[j] = 0.0f;
                    }
                    int ebr = eb[0];
#pragma unroll
                    for (int m = 1; m < E::NEB; ++m)
                        if ((blk >> 1) == m) ebr = eb[m];
#pragma unroll
                    for (int st = 0; st < 16 / T3_EG; ++st) {
                        const int g = blk * (16 / T3_EG) + st;
                        const int gf = g + E::INFL - 1;
                        if (gf < NSTEP)
                            t3_fetch(p_row + gf * T3_EG * ld8, ld8, gf * T3_EG, flim,
                                     old[(st + E::INFL - 1) % E::INFL]);
                        const int cl = g * T3_EG;
                        t3_store(args, H + st * T3_EG, L + st * T3_EG, p_row + cl * ld8, ld8, cl,
                                 lim, fa, ea, ebr, cl & 31, old[st % E::INFL],
                                 pf_row + cl * ld8f, ld8f, to_f64);
                    }
#pragma unroll
                    for (int j = 0; j < E::COLS - 16; ++j) L[j] = L[j + 16];
                }
                ++local;
            }
            if (stop) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0 && args.info) set_info(args.info, -1);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}


// C = alpha (hi + lo) + beta C over the written entries of a chunked contraction.
__global__ void acc2_to_f64_kernel(const float2 *acc, int64_t M, int64_t N, double alpha,
                                   double beta, double *C, int64_t ldc, int lower,
                                   int64_t diag_off) {
    const int64_t c = blockIdx.x;  // columns on x: N can exceed the 65,535 limit of y
    const int64_t r = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    if (r >= M || c >= N) return;
    if (lower && r + diag_off < c) return;
    const float2 v = acc[r + c * M];
    // the conversions by integer operations, one FP64 add; alpha = +-1 by the sign bit
    double x = f32_to_f64(v.x) + f32_to_f64(v.y);
    if (alpha == -1.0) x = -x;
    else if (alpha != 1.0) x *= alpha;
    if (beta != 0.0) x = fma(beta, C[r + c * ldc], x);
    C[r + c * ldc] = x;
}

// ---------------------------------------------------------------------------
// host side: tensor maps and launch
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D map over a slice store [S][rows][Kld]; one box is box_rows x 64 of
// box_slices consecutive slices (1, or every slice for the three-slice kernel).
static int make_slice_map(CUtensorMap *map, const TcOperand &op, int box_rows, int box_slices) {
    auto fn = encode_fn();
    if (!fn) return GP_ERR_CUDA;
    if ((reinterpret_cast<uintptr_t>(op.slices) & 15) || (op.Kld % TC_BK)) return GP_ERR_INVALID;
    cuuint64_t dims[3] = {(cuuint64_t)op.Kld, (cuuint64_t)op.rows, (cuuint64_t)op.S};
    cuuint64_t strides[2] = {(cuuint64_t)op.Kld * 2, (cuuint64_t)(op.rows * op.Kld * 2)};
    cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, (cuuint32_t)box_slices};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        op.S == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(map, dt, 3, const_cast<uint16_t *>(op.slices), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GP_OK : GP_ERR_CUDA;
}

static int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 0;
    }
    return n;
}

int tc_gemm(const TcOperand &A, const TcOperand &B, int64_t M, int64_t N, int64_t K,
            const TcOut &out, int tri_k, int64_t tri_off, int64_t *info, cudaStream_t s) {
    if (M <= 0 || N <= 0) return GP_OK;
    if (K % TC_BK || A.k_off % TC_BK || B.k_off % TC_BK) return GP_ERR_INVALID;
    if (A.k_off + K > A.Kld || B.k_off + K > B.Kld || A.S != B.S || (A.S != 3 && A.S != 5))
        return GP_ERR_INVALID;
    // normalized (three-slice) stores carry their row exponents; chunks of
    // both operands must line up with the stores' 512-column chunks
    const bool normalized = A.S == 3;
    if (normalized && (!A.ex || !B.ex)) return GP_ERR_INVALID;
    // one chunk width for both operands: 512, or 1024 for three-slice stores
    const int64_t kch = A.kch;
    if (B.kch != kch || !(kch == TC_CHUNK_K || (kch == 2 * TC_CHUNK_K && A.S == 3)))
        return GP_ERR_INVALID;
    if (A.k_off % kch || B.k_off % kch) return GP_ERR_INVALID;
    // the shared-memory opt-in is per device (setting it twice is harmless)
    // set once per device; a race between host threads only repeats the
    // (idempotent) attribute call
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
    if (!attr_set[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(tc_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(tc_gemm_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(tc_gemm3_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 T3_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(tc_gemm3_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 T3_SMEM) != cudaSuccess)
            return GP_ERR_CUDA;
        attr_set[dev].store(true, std::memory_order_release);
    }
    // three slices: the per-group kernel, whose stages carry every slice
    const bool three = A.S == 3;
    CUtensorMap ma, mb;
    GP_TRY(make_slice_map(&ma, A, TC_BM, three ? 3 : 1));
    GP_TRY(make_slice_map(&mb, B, TC_BN, three ? 3 : 1));
    TcGemmArgs a{};
    a.C = out.C;
    a.ldc = out.ldc;
    a.out_mode = out.mode;
    a.alpha = out.alpha;
    a.beta = out.beta;
    a.lower = out.lower;
    a.diag_off = out.diag_off;
    a.M = M;
    a.N = N;
    a.a_row_off = (int)A.row_off;
    a.b_row_off = (int)B.row_off;
    a.a_k_off = (int)A.k_off;
    a.b_k_off = (int)B.k_off;
    a.kblocks = (int)(K / TC_BK);
    a.tri_k = tri_k;
    a.tri_off = tri_off;
    a.kchunk = 0;
    a.idesc = idesc_f16kind_f32(TC_BM, TC_BN, !normalized);
    a.ex_a = normalized ? A.ex : nullptr;
    a.ex_b = normalized ? B.ex : nullptr;
    a.ex_ld_a = A.ex_ld;
    a.ex_ld_b = B.ex_ld;
    // Deep contractions: the operands' row bounds (and, normalized, their
    // scales) change every 512 columns of K, so the accumulators are flushed
    // per chunk: double-float outputs take each chunk directly, FP64 outputs
    // through the double-float buffer acc2.
    a.kch = (int)kch;
    const bool deep = K > kch;
    const bool via_acc2 = deep && out.mode == 0;
    // the three-slice kernel writes the FP64 result from the last chunk itself
    // (no zeroing of acc2 before, no conversion pass after) when beta = 0
    const bool fused = via_acc2 && A.S == 3 && out.beta == 0.0;
    if (deep) a.kchunk = (int)(kch / TC_BK);
    if (via_acc2) {
        if (!out.acc2) return GP_ERR_INVALID;
        if (N > 0x7fffffffLL || ceil_div(M, 256) > 65535) return GP_ERR_INVALID;
        a.out_mode = 2;
        a.C = out.acc2;
        a.ldc = M;
        a.alpha = 1.0;
        a.beta = 0.0;
        if (fused) {
            a.fuse_f64 = 1;
            a.Cf = static_cast<double *>(out.C);
            a.ldcf = out.ldc;
            a.alpha_f64 = out.alpha;
        } else if (cudaMemsetAsync(out.acc2, 0, sizeof(float2) * (size_t)M * (size_t)N, s) !=
                   cudaSuccess) {
            return GP_ERR_CUDA;
        }
    }
    a.tiles_m = (int)ceil_div(M, TC_BM);
    a.tiles_n = (int)ceil_div(N, TC_BN);
    a.info = info;
    // slice pairs grouped by accumulator.  With three slices the leading pair
    // owns the exact "hi" accumulator and the rest share "lo" (two tile
    // buffers); with more (integer slices) the groups d = 0, 1, 2 get one
    // accumulator each and d >= 3 a fourth (one buffer).  Within a shared
    // accumulator the groups go in order of increasing size (largest d
    // first): the tensor core aligns each step's products to the largest
    // exponent present and drops the bits below its window, so small
    // products added onto an already large running sum lose a systematic
    // share (the diagonal of a SYRK, where s1 s1 > 0, came out low by ~1e-8
    // relative); added first, they lose only what the later large ones cut.
    a.nacc = A.S >= 4 ? 4 : 2;
    a.nbuf = a.nacc * 2 <= 4 ? 2 : 1;
    int np = 0;
    for (int acc = 0; acc < a.nacc; ++acc) {
        const int dlo = acc, dhi = acc == a.nacc - 1 ? A.S - 1 : acc;
        for (int d = dhi; d >= dlo; --d)
            for (int p = 0; p <= d; ++p) {
                if (np >= TC_MAX_PAIRS) return GP_ERR_INVALID;
                a.pa[np] = p;
                a.pb[np] = d - p;
                a.acc_of[np] = acc;
                a.first_of[np] = (np == 0 || a.acc_of[np - 1] != acc) ? 1 : 0;
                ++np;
            }
    }
    a.npairs = np;
    const int64_t ntiles = (int64_t)a.tiles_m * a.tiles_n;
    const int sms = num_sms();
    int grid = (int)(ntiles < sms ? ntiles : (sms > 0 ? sms : 148));
    if (out.max_ctas > 0 && grid > out.max_ctas) grid = out.max_ctas;
    const int ev = prof_start(s);
    if (three && deep)
        tc_gemm3_kernel<8><<<grid, T3Epi<8>::THREADS, T3_SMEM, s>>>(ma, mb, a);
    else if (three)
        tc_gemm3_kernel<16><<<grid, T3Epi<16>::THREADS, T3_SMEM, s>>>(ma, mb, a);
    else if (a.nacc == 4)
        tc_gemm_kernel<4><<<grid, TC_THREADS, TC_SMEM, s>>>(ma, mb, a);
    else
        tc_gemm_kernel<2><<<grid, TC_THREADS, TC_SMEM, s>>>(ma, mb, a);
    GP_LAUNCH_CHECK();
    if (via_acc2 && !fused) {
        dim3 g2((unsigned)N, (unsigned)ceil_div(M, 256));
        acc2_to_f64_kernel<<<g2, 256, 0, s>>>(static_cast<const float2 *>(out.acc2), M, N,
                                               out.alpha, out.beta,
                                               static_cast<double *>(out.C), out.ldc, out.lower,
                                               out.diag_off);
        GP_LAUNCH_CHECK();
    }
    if (ev >= 0) {
        // slice-product flops over the useful output entries and K ranges
        double useful = 0.0;
        for (int64_t c = 0; c < N; ++c) {
            int64_t rows = M;
            if (out.lower) {
                const int64_t r_lo = c - out.diag_off;  // first row written in column c
                rows = r_lo <= 0 ? M : (r_lo >= M ? 0 : M - r_lo);
            }
            int64_t keff = K;
            if (tri_k && c - tri_off > 0) keff = K - (c - tri_off) > 0 ? K - (c - tri_off) : 0;
            useful += (double)rows * (double)keff;
        }
        prof_stop(ev, s, prof_contract_class(), 2.0 * np * useful, 0.0);
    }
    return GP_OK;
}

}  // namespace gp
