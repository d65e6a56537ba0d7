// batch_dag_tc.cu -- the mixed form of the batched task-graph launch: the
// same owner-computes tile tasks as the FP64 form (batch_dag.cu), on
// 128 x 128 tiles, with every tile contraction on the tcgen05 tensor cores.
//
// Operands are FP16 slice triples (the normalized three-slice encoding of
// the mixed form: per row of a tile, x 2^{7-e} = s0 + s1 + s2 with s0 an
// integer in [-128, 128], |x| < 2^e over the row), written once by the task
// that produces the tile, in both orientations (rows of the tile as K-major
// rows, and columns of the tile as K-major rows), so that every later
// contraction reads them verbatim:
//   CHOL(i, j)   A'_ij = C_ij - sum_k L_ik L_jk^T   (rows of L_ik, rows of L_jk)
//                L_ij = A'_ij W_j^T                 (rows of A', rows of W_j)
//   TRTRI(i, k)  P = sum_m X_im L_mk                (rows of X_im, columns of L_mk)
//                X_ik = -P W_k                      (rows of P, columns of W_k)
//   LG(i, j)     W_ij = sum_m X_mi^T X_mj           (columns of X_mi, columns of X_mj)
// One contraction step (a 128 x 128 x 128 tile product) is six slice pairs
// p + q < 3 in two TMEM accumulators: "hi" (s0 s0', integer sums below 2^21,
// exact) and "lo" (the rest, largest p + q first), 48 MMAs of 128 x 128 x 16.
// The step's two accumulators are scaled by 2^{e_a + e_b - 14} (row
// exponents of the two operand tiles) and added, in double-float on the
// FP32 pipe, to a running sum kept in the other half of TMEM; the next
// step's operands are copied into shared memory (cp.async) while this runs.
//
// FP64 stays where the method asks for it: the diagonal tile's Cholesky
// factor and inverse (four 64 x 64 blocks, FP64 CUDA cores), log det, the
// refinement residual's accumulation and the gradient's final sums.  The
// covariance entries (fill, residual, gradient) are evaluated in
// double-float.  The refinement of alpha (RES / CORR tasks) computes
// s = r - C alpha matrix-free and corrects alpha with FP32 solves by the
// low-precision factor (L_ij and W_j kept in FP32 for them); the residual
// it reports is the FP64-grade one.
#include "batch_dag.h"

#include <cuda_fp16.h>

#include <atomic>

namespace gp {

constexpr int QTHREADS = 256;
constexpr double QREFINE_TOL = 1e-11;

// shared memory (after aligning the base to 1 KB)
constexpr int QS_OPA = 0;
constexpr int QS_OPB = QOPER;
constexpr int QS_EXA = 2 * QOPER;          // int [2][128]
constexpr int QS_EXB = QS_EXA + 1024;      // int [2][128]
constexpr int QS_TAB = QS_EXB + 1024;      // float2 [256]
constexpr int QS_X = QS_TAB + 2048;        // float4 [128] column points
constexpr int QS_AV = QS_X + 2048;         // float2 [128] column alphas
constexpr int QS_RED = QS_AV + 1024;       // double [4][128]
constexpr int QS_EMAX = QS_RED + 4096;     // float [2][128]
constexpr int QS_MISC = QS_EMAX + 1024;    // mbarrier, TMEM slot, flags
constexpr int QS_BYTES = QS_MISC + 256;
constexpr int QS_DYN = QS_BYTES + 1024;    // + alignment slack
constexpr int QSTG_LD = QB + 1;            // staged double-float tile: float2 [128][129]
static_assert(QB * QSTG_LD * 8 <= 2 * QOPER, "staging tile exceeds the operand buffers");
static_assert(sizeof(DagSmem) <= 2 * QOPER, "FP64 overlay exceeds the operand buffers");

struct TcCtx {
    uint8_t *opA, *opB;
    int *exA, *exB;
    float2 *tab;
    float4 *xs;
    float2 *av;
    double *red;
    float *emax;
    uint64_t *mbar;
    int *ok;
    int *misc;
    uint32_t tmem;
    uint32_t phase;
    double *scr;
    DagHdr *h;
};

// flag layout of a mixed problem (see dag_nflags)
__device__ __forceinline__ int *f_L(const DagProb &P) { return P.flag; }
__device__ __forceinline__ int *f_X(const DagProb &P) { return P.flag + dag_ntiles(P.T); }
__device__ __forceinline__ int *f_solved(const DagProb &P) { return P.flag + dag_solved_flag(P.T); }
__device__ __forceinline__ int *f_res(const DagProb &P, int e) { return f_solved(P) + 1 + e; }
__device__ __forceinline__ int *f_corr(const DagProb &P, int e) {
    return f_solved(P) + 1 + DAG_EVALS + e;
}
__device__ __forceinline__ int *f_fin(const DagProb &P) { return f_solved(P) + 2 * DAG_EVALS; }
__device__ __forceinline__ int *f_lg(const DagProb &P) { return P.flag + dag_lg_flag(P.T, 1); }
__device__ __forceinline__ int *f_conv(const DagProb &P) { return f_lg(P) + 1; }

__device__ __forceinline__ const uint8_t *store_tile(const uint8_t *base, int T, int i, int j) {
    return base + (size_t)tile_index(T, i, j) * QSTRIDE;
}
__device__ __forceinline__ float *l32_tile(const DagProb &P, int i, int j) {
    return P.L32 + (size_t)tile_index(P.T, i, j) * (QB * QB);
}

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// bound exponent of a row / column with largest magnitude m: |x| < 2^e
__device__ __forceinline__ int bound_exp(float m) {
    int e = 0;
    if (m > 0.0f) frexpf(m, &e);
    return max(-100, min(e, 120));
}

// three normalized FP16 slices of v (a double-float) at scale sc = 2^{7-e}
__device__ __forceinline__ void split3_df(dfl v, float sc, uint16_t &s0, uint16_t &s1,
                                          uint16_t &s2) {
    const float yh = __fmul_rn(v.h, sc), yl = __fmul_rn(v.l, sc);
    const float q = rintf(yh);
    const dfl t = df_two_sum(__fsub_rn(yh, q), yl);  // yh - q is exact
    const __half h1 = __float2half_rn(t.h);
    const float rest = __fadd_rn(__fsub_rn(t.h, __half2float(h1)), t.l);  // t.h - h1 exact
    s0 = __half_as_ushort(__float2half_rn(q));
    s1 = __half_as_ushort(h1);
    s2 = __half_as_ushort(__float2half_rn(rest));
}

__device__ __forceinline__ dfl d2df(double v) {
    return f64_to_df(static_cast<unsigned long long>(__double_as_longlong(v)));
}

// global writes of this CTA visible to its own later L2 reads
__device__ __forceinline__ void cta_gsync() {
    __threadfence();
    __syncthreads();
}

// --------------------------------------------------------------------------
// the tile contraction engine
// --------------------------------------------------------------------------
__device__ __forceinline__ void tc_load(uint8_t *dst, int *ex_dst, const uint8_t *src) {
    for (int e = threadIdx.x; e < QOPER / 16; e += QTHREADS) cp_async16(dst + 16 * e, src + 16 * e);
    if (threadIdx.x < 32) cp_async16(ex_dst + 4 * threadIdx.x, src + QOPER + 16 * threadIdx.x);
}

// 48 MMAs of one 128 x 128 x 128 step: hi (TMEM columns 0-127) = s0 s0',
// lo (128-255) = pairs with p + q = 2, then p + q = 1.
__device__ void tc_issue(const TcCtx &c) {
    constexpr uint32_t idesc = idesc_f16kind_f32(QB, QB, false);
    const int PA[6] = {0, 0, 1, 2, 0, 1}, PB[6] = {0, 2, 1, 0, 1, 0};
    const uint32_t a0 = smem_u32(c.opA), b0 = smem_u32(c.opB);
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        const uint32_t acc = c.tmem + (p == 0 ? 0u : (uint32_t)QB);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t off = h * QATOM + kk * 32;
                mma_f16_ss(acc, sdesc_sw128(a0 + PA[p] * QSLICE + off),
                           sdesc_sw128(b0 + PB[p] * QSLICE + off), idesc,
                           (p <= 1 && h == 0 && kk == 0) ? 0u : 1u);
            }
    }
    mma_commit(c.mbar);
    if (c.h->prof) atomicAdd(&c.h->steps, 1ull);
}

// Every thread waits for the step's MMAs (bounded; a second bounded wait
// after a timeout, so that no MMA is in flight when the CTA leaves).
__device__ bool tc_mma_wait(TcCtx &c, const DagProb &P) {
    bool ok = mbar_wait(c.mbar, c.phase);
    if (!ok) {
        mbar_wait(c.mbar, c.phase);
        if (threadIdx.x == 0) {
            set_info(P.info, -1);
            atomicExch(&c.h->abort, 1);
        }
    }
    c.phase ^= 1u;
    tc_fence_after();
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// running (TMEM 256-511: hi parts, lo parts) (+)= (hi + lo) 2^{ea + eb - 14}
__device__ void tc_drain(const TcCtx &c, int buf, bool first) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = w & 3, ch = w >> 2;
    const int row = qd * 32 + lane;
    const float fa = pow2f(c.exA[buf * QB + row] - 7);
    const uint32_t tb = c.tmem + ((uint32_t)(qd * 32) << 16);
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
        const int col0 = ch * 64 + g * 16;
        uint32_t hi[16], lo[16], rh[16], rl[16];
        tmem_ld_32x32b_x16(tb + col0, hi);
        tmem_ld_32x32b_x16(tb + QB + col0, lo);
        if (!first) {
            tmem_ld_32x32b_x16(tb + 2 * QB + col0, rh);
            tmem_ld_32x32b_x16(tb + 3 * QB + col0, rl);
        }
        tmem_ld_wait();
        // the step's hi part (an exact integer sum times a power of two) goes
        // in through one double-float add, the lo part (below 2^-8 of it)
        // straight into the low word: its rounding there is below 2^-48 of
        // the running value
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float f = __fmul_rn(fa, pow2f(c.exB[buf * QB + col0 + j] - 7));
            const float a = __fmul_rn(__uint_as_float(hi[j]), f);
            const float b = __fmul_rn(__uint_as_float(lo[j]), f);
            dfl v;
            if (first) {
                v = df_two_sum(a, b);
            } else {
                v = df_add_f(dfl{__uint_as_float(rh[j]), __uint_as_float(rl[j])}, a);
                v.l = __fadd_rn(v.l, b);
            }
            rh[j] = __float_as_uint(v.h);
            rl[j] = __float_as_uint(v.l);
        }
        tmem_st_32x32b_x16(tb + 2 * QB + col0, rh);
        tmem_st_32x32b_x16(tb + 3 * QB + col0, rl);
    }
    tmem_st_wait();
}

// sum over q < Q of the step products of pair(q) into the running sum.
// pair(q, a, b) waits for step q's operands and names their stores.
template <class F>
__device__ bool tc_contract(TcCtx &c, const DagProb &P, int Q, F pair) {
    const uint8_t *ga = nullptr, *gb = nullptr;
    if (!pair(0, ga, gb)) return false;
    tc_load(c.opA, c.exA, ga);
    tc_load(c.opB, c.exB, gb);
    cp_async_commit();
    for (int q = 0; q < Q; ++q) {
        const int buf = q & 1;
        cp_async_wait_all();
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            tc_issue(c);
        }
        if (!tc_mma_wait(c, P)) return false;
        if (q + 1 < Q) {
            if (!pair(q + 1, ga, gb)) return false;
            tc_load(c.opA, c.exA + QB * (buf ^ 1), ga);
            tc_load(c.opB, c.exB + QB * (buf ^ 1), gb);
            cp_async_commit();
        }
        tc_drain(c, buf, q == 0);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    return true;
}

// One step whose A operand is already in opA / exA[0] (written by this
// CTA's threads) and whose B operand is the store gb; the product lands in
// the running sum (overwritten).
__device__ bool tc_single(TcCtx &c, const DagProb &P, const uint8_t *gb) {
    tc_load(c.opB, c.exB, gb);
    cp_async_commit();
    cp_async_wait_all();
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        tc_issue(c);
    }
    if (!tc_mma_wait(c, P)) return false;
    tc_drain(c, 0, true);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return true;
}

// Read 16 columns of the running sum (this thread's row).
__device__ __forceinline__ void run_ld16(const TcCtx &c, int col0, dfl (&v)[16]) {
    const int w = threadIdx.x >> 5, qd = w & 3;
    const uint32_t tb = c.tmem + ((uint32_t)(qd * 32) << 16);
    uint32_t rh[16], rl[16];
    tmem_ld_32x32b_x16(tb + 2 * QB + col0, rh);
    tmem_ld_32x32b_x16(tb + 3 * QB + col0, rl);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = dfl{__uint_as_float(rh[j]), __uint_as_float(rl[j])};
}

// --------------------------------------------------------------------------
// FP64 scratch tile (block-major 64 x 64 blocks: element (r, c) of a
// 128 x 128 tile at block (r / 64) + 2 (c / 64), offset (r % 64) + 64 (c % 64))
// --------------------------------------------------------------------------
__device__ __forceinline__ int scr_idx(int r, int c) {
    return (((r >> 6) + 2 * (c >> 6)) << 12) + (r & 63) + 64 * (c & 63);
}

// Slice the rows of the scratch tile into opA / exA[0] (row exponents from
// c.emax, the per-half row maxima of |hi|).
__device__ void scr_rows_to_opA(TcCtx &c) {
    const int t = threadIdx.x, r = t & (QB - 1), h = t >> 7;
    const float m = fmaxf(c.emax[r], c.emax[QB + r]);
    const int e = bound_exp(m);
    if (h == 0) c.exA[r] = e;
    const float sc = pow2f(7 - e);
    for (int cc = 0; cc < 8; ++cc) {
        uint16_t s[3][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int col = 64 * h + 8 * cc + u;
            split3_df(d2df(__ldcg(c.scr + scr_idx(r, col))), sc, s[0][u], s[1][u], s[2][u]);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            uint4 v;
            v.x = s[p][0] | ((uint32_t)s[p][1] << 16);
            v.y = s[p][2] | ((uint32_t)s[p][3] << 16);
            v.z = s[p][4] | ((uint32_t)s[p][5] << 16);
            v.w = s[p][6] | ((uint32_t)s[p][7] << 16);
            *reinterpret_cast<uint4 *>(c.opA + p * QSLICE + h * QATOM + r * 128 +
                                       ((cc ^ (r & 7)) << 4)) = v;
        }
    }
}

// Write the staged double-float tile stg[r][c] as slice stores (rows ->
// rowst, columns -> colst) and optionally as FP32 (column-major).
__device__ void write_outputs(TcCtx &c, const float2 *stg, uint8_t *rowst, uint8_t *colst,
                              float *f32) {
    const int t = threadIdx.x, a = t & (QB - 1), h = t >> 7;
    // rows: thread (row a, columns 64h..)
    float m = 0.0f;
    for (int u = 0; u < 64; ++u) m = fmaxf(m, fabsf(stg[a * QSTG_LD + 64 * h + u].x));
    c.emax[h * QB + a] = m;
    __syncthreads();
    {
        const int e = bound_exp(fmaxf(c.emax[a], c.emax[QB + a]));
        if (h == 0) reinterpret_cast<int *>(rowst + QOPER)[a] = e;
        const float sc = pow2f(7 - e);
        for (int cc = 0; cc < 8; ++cc) {
            uint16_t s[3][8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int col = 64 * h + 8 * cc + u;
                const float2 v = stg[a * QSTG_LD + col];
                split3_df(dfl{v.x, v.y}, sc, s[0][u], s[1][u], s[2][u]);
                if (f32) f32[a + QB * col] = v.x;
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                uint4 v;
                v.x = s[p][0] | ((uint32_t)s[p][1] << 16);
                v.y = s[p][2] | ((uint32_t)s[p][3] << 16);
                v.z = s[p][4] | ((uint32_t)s[p][5] << 16);
                v.w = s[p][6] | ((uint32_t)s[p][7] << 16);
                *reinterpret_cast<uint4 *>(rowst + p * QSLICE + h * QATOM + a * 128 +
                                           ((cc ^ (a & 7)) << 4)) = v;
            }
        }
    }
    __syncthreads();
    // columns: thread (column a, rows 64h..)
    m = 0.0f;
    for (int u = 0; u < 64; ++u) m = fmaxf(m, fabsf(stg[(64 * h + u) * QSTG_LD + a].x));
    c.emax[h * QB + a] = m;
    __syncthreads();
    {
        const int e = bound_exp(fmaxf(c.emax[a], c.emax[QB + a]));
        if (h == 0) reinterpret_cast<int *>(colst + QOPER)[a] = e;
        const float sc = pow2f(7 - e);
        for (int rr = 0; rr < 8; ++rr) {
            uint16_t s[3][8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float2 v = stg[(64 * h + 8 * rr + u) * QSTG_LD + a];
                split3_df(dfl{v.x, v.y}, sc, s[0][u], s[1][u], s[2][u]);
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                uint4 v;
                v.x = s[p][0] | ((uint32_t)s[p][1] << 16);
                v.y = s[p][2] | ((uint32_t)s[p][3] << 16);
                v.z = s[p][4] | ((uint32_t)s[p][5] << 16);
                v.w = s[p][6] | ((uint32_t)s[p][7] << 16);
                *reinterpret_cast<uint4 *>(colst + p * QSLICE + h * QATOM + a * 128 +
                                           ((rr ^ (a & 7)) << 4)) = v;
            }
        }
    }
}

// running sum (times sgn) -> stg (this thread's row, 64 columns)
__device__ void run_to_stg(const TcCtx &c, float2 *stg, float sgn) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = w & 3, ch = w >> 2;
    const int row = qd * 32 + lane;
    for (int g = 0; g < 4; ++g) {
        dfl v[16];
        run_ld16(c, ch * 64 + g * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            stg[row * QSTG_LD + ch * 64 + g * 16 + j] = make_float2(sgn * v[j].h, sgn * v[j].l);
    }
}

// running sum (or -(C - running) style values given by fn) -> FP64 scratch
// and per-half row maxima of |hi| in c.emax.
template <class F>
__device__ void tile_to_scr(TcCtx &c, F value) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = w & 3, ch = w >> 2;
    const int row = qd * 32 + lane;
    float m = 0.0f;
    for (int g = 0; g < 4; ++g) {
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
            const int col = ch * 64 + g * 16 + j;
            const dfl v = value(row, col, g, j);
            m = fmaxf(m, fabsf(v.h));
            c.scr[scr_idx(row, col)] = df_to_double(v);
        }
    }
    c.emax[ch * QB + row] = m;
}

// --------------------------------------------------------------------------
// tasks
// --------------------------------------------------------------------------
__device__ void stage_points(TcCtx &c, const DagProb &P, int tile) {
    if (threadIdx.x < QB) {
        const int64_t g = (int64_t)tile * QB + threadIdx.x;
        const double2 p = g < P.n ? P.x[g] : make_double2(0.0, 0.0);
        // a location that is not finite: d_info = -2 (first status wins)
        if (!isfinite(p.x) || !isfinite(p.y)) set_info(P.info, -2);
        c.xs[threadIdx.x] = df_point(p);
    }
}

// ---------------------------------------------------------------------------
// The diagonal tile in double-float (FP32 pairs): the FP64 pipe of this part
// runs at 1/64 of the FP32 rate, and the 64 x 64 blocks of the diagonal tile
// (their factors, inverses and products) took most of the FP64 work of the
// batched launch.  The pairs carry about 48 bits, the FP64 scratch blocks
// stay the interface (converted by integer operations on load, one FP64 add
// per entry on store).
// ---------------------------------------------------------------------------
__device__ __forceinline__ dfl ld_df(const double *p) {
    return f64_to_df(static_cast<unsigned long long>(__double_as_longlong(__ldcg(p))));
}

// stage_a / stage_b of a 64 x 64 FP64 block as double-float pairs
template <int TA>
__device__ __forceinline__ void stage_a_df(const double *A, dfl *sA) {
    for (int e = threadIdx.x; e < DB * DB; e += DAG_THREADS) {
        const dfl v = ld_df(A + e);
        const int lo = e & (DB - 1), hi = e >> 6;
        if (TA == 0) sA[hi * DLD + lo] = v;
        else sA[lo * DLD + hi] = v;
    }
}

template <int TB>
__device__ __forceinline__ void stage_b_df(const double *B, dfl *sB) {
    for (int e = threadIdx.x; e < DB * DB; e += DAG_THREADS) {
        const dfl v = ld_df(B + e);
        const int lo = e & (DB - 1), hi = e >> 6;
        if (TB == 0) sB[lo * DLD + hi] = v;
        else sB[hi * DLD + lo] = v;
    }
}

// (h, l) += a b with the product's error terms and the sum's rounding error
// gathered in l (renormalized once at the end of a product).
__device__ __forceinline__ void df_acc(float &h, float &l, dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float pe = __fmaf_rn(a.h, b.h, -p);
    pe = __fmaf_rn(a.h, b.l, pe);
    pe = __fmaf_rn(a.l, b.h, pe);
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, pe));
}

// 64 x 64 product on staged double-float operands (sA [t][r], sB [t][c])
// with a blocked thread mapping: acc (rows 4 tx + a, columns 4 ty + b) +/-=
// sum over t in [tlo, thi) of sA[t][r] sB[t][c].  The diagonal tile's
// products have triangular factors, and a thread skips the t range where its
// factor block vanishes.
template <bool NEG>
__device__ __forceinline__ void blk_mma_df(float (&ah)[4][4], float (&al)[4][4], const dfl *sA,
                                           const dfl *sB, int tlo, int thi) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 2
    for (int t = tlo; t < thi; ++t) {
        dfl av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            av[a] = sA[t * DLD + 4 * tx + a];
            if (NEG) av[a] = df_neg(av[a]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = sB[t * DLD + 4 * ty + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) df_acc(ah[a][b], al[a][b], av[a], bv[b]);
    }
}

__device__ __forceinline__ void acc_zero_df(float (&ah)[4][4], float (&al)[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ah[a][b] = al[a][b] = 0.0f;
}

// the block of blk_mma_df into the FP64 block G (ld 64)
__device__ __forceinline__ void blk_store_df(const float (&ah)[4][4], const float (&al)[4][4],
                                             double *G) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a)
            G[(4 * tx + a) + DB * (4 * ty + b)] = df_to_double(df_quick_sum(ah[a][b], al[a][b]));
}

// potrf_inv_tile in double-float: the 64 x 64 block staged (as pairs) in
// sm.sA is factored (right-looking, the unscaled form a_rc -= a_rj a_cj /
// a_jj, then L_rc = a_rc / sqrt(a_cc)); L is written to G and W = L^{-1} to
// Wg (FP64, ld 64), and the block's log-det share to *logpart.  Pivots that
// are not positive are reported as in potrf_inv_tile.
__device__ void potrf_inv_tile_df(const DagProb &P, int j, double *G, double *Wg,
                                  double *logpart, DagSmem &sm) {
    const int tid = threadIdx.x;
    dfl *S = reinterpret_cast<dfl *>(sm.sA);
    dfl *Y = reinterpret_cast<dfl *>(sm.sB);
    dfl *dinv = reinterpret_cast<dfl *>(sm.dinv);
    dfl *lj = reinterpret_cast<dfl *>(sm.lj);
    if (tid == 0) {
        sm.bad = 0;
        sm.badcol = 0;
    }
    __syncthreads();
    for (int jj = 0; jj < DB; ++jj) {
        const dfl *cj = S + jj * DLD;
        if (tid < DB) {
            const dfl d = cj[jj];
            if (!(d.h > 0.0f)) {
                if (tid == 0) {
                    sm.bad = 1;
                    sm.badcol = jj;
                }
            } else {
                const dfl inv = df_rcp(d);
                if (tid == 0) dinv[jj] = inv;
                if (tid > jj) lj[tid] = df_mul(cj[tid], inv);
            }
        }
        __syncthreads();
        if (sm.bad) break;
        const int ntri = (DB - 1 - jj) * (DB - jj) / 2;
        for (int e = tid; e < ntri; e += DAG_THREADS) {
            int r, c;
            tri_desc_entry(e, DB, r, c);
            S[c * DLD + r] = df_fms(S[c * DLD + r], cj[r], lj[c]);
        }
        __syncthreads();
    }
    if (sm.bad) {
        if (tid == 0) set_info(P.info, (int64_t)j * DB + sm.badcol + 1);
        return;
    }
    if (tid < DB) dinv[tid] = df_sqrt(dinv[tid]);
    __syncthreads();
    for (int e = tid; e < DB * DB; e += DAG_THREADS) {
        const int r = e & (DB - 1), c = e >> 6;
        const dfl v = (r >= c) ? df_mul(S[c * DLD + r], dinv[c]) : dfl{0.0f, 0.0f};
        S[c * DLD + r] = v;
        G[e] = df_to_double(v);
    }
    __syncthreads();
    if (tid < DB) {
        const dfl d = S[tid * DLD + tid];
        lj[tid] = df_rcp(d);  // 1 / L_rr
        sm.vr[tid] = ((int64_t)j * DB + tid < P.n) ? log(df_to_double(d)) : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int r = 0; r < DB; ++r) s += sm.vr[r];
        *logpart = s;
    }
    // W = L^{-1}: with Y = I and M_lc = L_lc / L_ll, for l descending,
    // Y_c -= Y_l M_lc (c < l); then W_c = Y_c / L_cc (columns).
    for (int e = tid; e < DB * DB; e += DAG_THREADS) {
        const int r = e & (DB - 1), c = e >> 6;
        if (r > c) S[c * DLD + r] = df_mul(S[c * DLD + r], lj[r]);
        Y[c * DLD + r] = dfl{(r == c) ? 1.0f : 0.0f, 0.0f};
    }
    __syncthreads();
    for (int l = DB - 1; l > 0; --l) {
        const int nr = DB - l;
        for (int e = tid; e < l * nr; e += DAG_THREADS) {
            const int c = e / nr, r = l + (e - c * nr);
            Y[c * DLD + r] = df_fms(Y[c * DLD + r], Y[l * DLD + r], S[c * DLD + l]);
        }
        __syncthreads();
    }
    for (int e = tid; e < DB * DB; e += DAG_THREADS) {
        const int r = e & (DB - 1), c = e >> 6;
        Wg[e] = (r >= c) ? df_to_double(df_mul(Y[c * DLD + r], lj[c])) : 0.0;
    }
}

// Factor and inverse of the diagonal tile held in the FP64 scratch (blocks
// 0 = A11, 1 = A21, 3 = A22), in double-float: L11, W11; L21 = A21 W11^T;
// L22, W22 from A22 - L21 L21^T (lower half); W21 = -W22 (L21 W11).
// Returns the tile's log-det share.
__device__ double diag_factor(TcCtx &c, const DagProb &P, int j) {
    DagSmem &dsm = *reinterpret_cast<DagSmem *>(c.opA);
    dfl *sA = reinterpret_cast<dfl *>(dsm.sA), *sB = reinterpret_cast<dfl *>(dsm.sB);
    double *B = c.scr;
    const int D = 64 * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double *ld = c.red;  // two shares
    float ah[4][4], al[4][4];
    __syncthreads();
    stage_a_df<0>(B + 0 * D, sA);
    __syncthreads();
    potrf_inv_tile_df(P, 2 * j, B + 0 * D, B + 4 * D, ld + 0, dsm);
    cta_gsync();
    // L21 = A21 W11^T: W11(c, t) = 0 for t > c
    stage_a_df<0>(B + 1 * D, sA);
    stage_b_df<1>(B + 4 * D, sB);
    __syncthreads();
    acc_zero_df(ah, al);
    blk_mma_df<false>(ah, al, sA, sB, 0, 4 * ty + 4);
    blk_store_df(ah, al, B + 1 * D);
    cta_gsync();
    // A22 - L21 L21^T on the blocks that touch the lower half
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const dfl v = ld_df(B + 3 * D + (4 * tx + a) + 64 * (4 * ty + b));
            ah[a][b] = v.h;
            al[a][b] = v.l;
        }
    stage_a_df<0>(B + 1 * D, sA);
    stage_b_df<1>(B + 1 * D, sB);
    __syncthreads();
    if (tx >= ty) blk_mma_df<true>(ah, al, sA, sB, 0, DB);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            sA[(4 * ty + b) * DLD + 4 * tx + a] = df_quick_sum(ah[a][b], al[a][b]);
    __syncthreads();
    potrf_inv_tile_df(P, 2 * j + 1, B + 3 * D, B + 6 * D, ld + 1, dsm);
    cta_gsync();
    // L21 W11: W11(t, c) = 0 for t < c
    stage_a_df<0>(B + 1 * D, sA);
    stage_b_df<0>(B + 4 * D, sB);
    __syncthreads();
    acc_zero_df(ah, al);
    blk_mma_df<false>(ah, al, sA, sB, 4 * ty, DB);
    blk_store_df(ah, al, B + 2 * D);
    cta_gsync();
    // W21 = -W22 (L21 W11): W22(r, t) = 0 for t > r
    stage_a_df<0>(B + 6 * D, sA);
    stage_b_df<0>(B + 2 * D, sB);
    __syncthreads();
    acc_zero_df(ah, al);
    blk_mma_df<true>(ah, al, sA, sB, 0, 4 * tx + 4);
    blk_store_df(ah, al, B + 5 * D);
    cta_gsync();
    return ld[0] + ld[1];
}

__device__ bool tc_chol(TcCtx &c, const DagProb &P, int i, int j) {
    const int T = P.T;
    int *Lf = f_L(P), *Xf = f_X(P);
    const int tij = tile_index(T, i, j);
    if (!dag_failed(P)) {
        if (j > 0) {
            auto pair = [&](int k, const uint8_t *&ga, const uint8_t *&gb) -> bool {
                if (!dag_wait(Lf + tile_index(T, i, k), 1, c.h, P.info, c.ok)) return false;
                if (i != j && !dag_wait(Lf + tile_index(T, j, k), 1, c.h, P.info, c.ok)) return false;
                ga = store_tile(P.LSr, T, i, k);
                gb = store_tile(P.LSr, T, j, k);
                return true;
            };
            if (!tc_contract(c, P, j, pair)) return false;
        }
        // A' = C_ij - running, to the FP64 scratch
        __syncthreads();
        stage_points(c, P, i);  // checks the row tile's locations
        __syncthreads();
        stage_points(c, P, j);
        __syncthreads();
        {
            const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = w & 3, ch = w >> 2;
            const int row = qd * 32 + lane;
            const int64_t gi = (int64_t)i * QB + row;
            const float4 xi = df_point(gi < P.n ? P.x[gi] : make_double2(0.0, 0.0));
            const bool has_run = j > 0;
            dfl run[16];
            auto value = [&](int r, int col, int g, int jj) -> dfl {
                if (jj == 0 && has_run) run_ld16(c, ch * 64 + g * 16, run);
                const int64_t gc = (int64_t)j * QB + col;
                dfl v;
                if (gi >= P.n || gc >= P.n) v = dfl{gi == gc ? 1.0f : 0.0f, 0.0f};
                else if (gi == gc) v = P.ddiag;
                else {
                    dfl unused;
                    df_cov_s<false>(P.kind, P.dscale, P.ds2, df_dist(xi, c.xs[col]), c.tab, v, unused);
                }
                if (has_run) v = df_add(v, df_neg(run[jj]));
                return v;
            };
            tile_to_scr(c, value);
        }
        cta_gsync();
        if (i == j) {
            const double ldet = diag_factor(c, P, j);
            if (threadIdx.x == 0) P.part[j] = ldet;
            // W_j (blocks 4, 5, 6) -> stg -> stores (rows, columns, FP32)
            float2 *stg = reinterpret_cast<float2 *>(c.opA);
            __syncthreads();
            for (int e = threadIdx.x; e < QB * QB; e += QTHREADS) {
                const int r = e & (QB - 1), col = e >> 7;
                double v = 0.0;
                if (r >= 64 && col < 64) v = __ldcg(c.scr + 5 * 4096 + (r - 64) + 64 * col);
                else if (r < 64 && col < 64) v = __ldcg(c.scr + 4 * 4096 + r + 64 * col);
                else if (r >= 64 && col >= 64) v = __ldcg(c.scr + 6 * 4096 + (r - 64) + 64 * (col - 64));
                const dfl d = d2df(v);
                stg[r * QSTG_LD + col] = make_float2(d.h, d.l);
            }
            __syncthreads();
            write_outputs(c, stg, const_cast<uint8_t *>(store_tile(P.XSr, T, j, j)),
                          const_cast<uint8_t *>(store_tile(P.XSc, T, j, j)), l32_tile(P, j, j));
        } else {
            // L_ij = A' W_j^T
            scr_rows_to_opA(c);
            fence_proxy_async_smem();
            if (!dag_wait(Lf + tile_index(T, j, j), 1, c.h, P.info, c.ok)) return false;
            if (!tc_single(c, P, store_tile(P.XSr, T, j, j))) return false;
            float2 *stg = reinterpret_cast<float2 *>(c.opA);
            run_to_stg(c, stg, 1.0f);
            __syncthreads();
            write_outputs(c, stg, const_cast<uint8_t *>(store_tile(P.LSr, T, i, j)),
                          const_cast<uint8_t *>(store_tile(P.LSc, T, i, j)), l32_tile(P, i, j));
        }
    }
    dag_signal(Lf + tij);
    if (i == j) dag_signal(Xf + tij);
    return true;
}

__device__ bool tc_trtri(TcCtx &c, const DagProb &P, int i, int k) {
    const int T = P.T;
    int *Lf = f_L(P), *Xf = f_X(P);
    if (!dag_failed(P)) {
        auto pair = [&](int q, const uint8_t *&ga, const uint8_t *&gb) -> bool {
            const int m = i - q;  // m = i, i - 1, ..., k + 1
            if (!dag_wait(Xf + tile_index(T, i, m), 1, c.h, P.info, c.ok)) return false;
            if (!dag_wait(Lf + tile_index(T, m, k), 1, c.h, P.info, c.ok)) return false;
            ga = store_tile(P.XSr, T, i, m);
            gb = store_tile(P.LSc, T, m, k);
            return true;
        };
        if (!tc_contract(c, P, i - k, pair)) return false;
        {
            dfl run[16];
            const int ch = (threadIdx.x >> 5) >> 2;
            auto value = [&](int r, int col, int g, int jj) -> dfl {
                if (jj == 0) run_ld16(c, ch * 64 + g * 16, run);
                return run[jj];
            };
            tile_to_scr(c, value);
        }
        cta_gsync();
        scr_rows_to_opA(c);
        fence_proxy_async_smem();
        if (!dag_wait(Xf + tile_index(T, k, k), 1, c.h, P.info, c.ok)) return false;
        if (!tc_single(c, P, store_tile(P.XSc, T, k, k))) return false;
        float2 *stg = reinterpret_cast<float2 *>(c.opA);
        run_to_stg(c, stg, -1.0f);
        __syncthreads();
        write_outputs(c, stg, const_cast<uint8_t *>(store_tile(P.XSr, T, i, k)),
                      const_cast<uint8_t *>(store_tile(P.XSc, T, i, k)), nullptr);
    }
    dag_signal(Xf + tile_index(T, i, k));
    return true;
}

// FP32 solves by the low-precision factor: b <- L^{-T} L^{-1} b on the
// problem's padded vector (FP64 storage), tile rows with W_i on the diagonal.
// Every FP32 tile streams through two shared-memory buffers (cp.async,
// columns padded to 132 floats): the forward sweep reads tile columns
// (lanes = rows), the backward sweep tile rows as float4 (lanes = columns),
// both without bank conflicts.
constexpr int SLD = 132;                    // padded column stride (floats)
constexpr int SBUF = QB * SLD * 4;          // one staged tile (bytes)

__device__ __forceinline__ void stage_l32(float *dst, const float *src) {
    for (int e = threadIdx.x; e < QB * 32; e += QTHREADS) {
        const int col = e >> 5, q = e & 31;
        cp_async16(dst + col * SLD + 4 * q, src + col * QB + 4 * q);
    }
    cp_async_commit();
}

__device__ void lowp_solve(TcCtx &c, const DagProb &P, double *b, double *t) {
    const int T = P.T, tid = threadIdx.x, r = tid & (QB - 1), h = tid >> 7;
    float *buf0 = reinterpret_cast<float *>(c.opA), *buf1 = reinterpret_cast<float *>(c.opA + SBUF);
    float *red = reinterpret_cast<float *>(c.red);  // [2][128]
    float *tv = red + 2 * QB;                       // [128]
    // forward: t_i = W_i (b_i - sum_{j<i} L_ij t_j); steps j = 0..i-1, then W_i
    for (int i = 0; i < T; ++i) {
        float s = 0.0f;
        __syncthreads();
        stage_l32(buf0, l32_tile(P, i, i == 0 ? 0 : 0));
        for (int st = 0; st <= i; ++st) {
            float *cur = (st & 1) ? buf1 : buf0;
            if (st < i) {
                stage_l32((st & 1) ? buf0 : buf1, l32_tile(P, i, st + 1));
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                cp_async_wait_all();
            }
            __syncthreads();
            if (st < i) {
                const double *tj = t + (int64_t)st * QB;
#pragma unroll 8
                for (int col = 64 * h; col < 64 * h + 64; ++col) s = fmaf(cur[col * SLD + r], (float)tj[col], s);
            } else {
                red[h * QB + r] = s;
                __syncthreads();
                if (tid < QB) tv[tid] = (float)__ldcg(b + (int64_t)i * QB + tid) - (red[tid] + red[QB + tid]);
                __syncthreads();
                float u = 0.0f;
                for (int col = 64 * h; col < 64 * h + 64 && col <= r; ++col) u = fmaf(cur[col * SLD + r], tv[col], u);
                red[h * QB + r] = u;
                __syncthreads();
                if (tid < QB) t[(int64_t)i * QB + tid] = red[tid] + red[QB + tid];
            }
            __syncthreads();
        }
    }
    // backward: b_i = W_i^T (t_i - sum_{j>i} L_ji^T b_j); steps j = T-1..i+1, then W_i
    for (int i = T - 1; i >= 0; --i) {
        float s = 0.0f;
        const int nst = T - 1 - i;  // off-diagonal steps
        __syncthreads();
        stage_l32(buf0, l32_tile(P, nst > 0 ? T - 1 : i, i));
        for (int st = 0; st <= nst; ++st) {
            float *cur = (st & 1) ? buf1 : buf0;
            if (st < nst) {
                const int jn = T - 2 - st;  // next tile row: T-2, ..., i+1, then i (W_i)
                stage_l32((st & 1) ? buf0 : buf1, l32_tile(P, jn > i ? jn : i, i));
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                cp_async_wait_all();
            }
            __syncthreads();
            if (st < nst) {
                const int j = T - 1 - st;
                const double *bj = b + (int64_t)j * QB;
                // (L_ji^T b_j)[r] = sum_c L_ji(c, r) b_j(c): row r of the staged tile's transpose
                const float4 *col_r = reinterpret_cast<const float4 *>(cur + r * SLD + 64 * h);
#pragma unroll 4
                for (int q = 0; q < 16; ++q) {
                    const float4 v = col_r[q];
                    const int c0 = 64 * h + 4 * q;
                    s = fmaf(v.x, (float)bj[c0], s);
                    s = fmaf(v.y, (float)bj[c0 + 1], s);
                    s = fmaf(v.z, (float)bj[c0 + 2], s);
                    s = fmaf(v.w, (float)bj[c0 + 3], s);
                }
            } else {
                red[h * QB + r] = s;
                __syncthreads();
                if (tid < QB) tv[tid] = (float)t[(int64_t)i * QB + tid] - (red[tid] + red[QB + tid]);
                __syncthreads();
                // b_i(r) = sum_{c >= r} W_i(c, r) tv(c)
                float u = 0.0f;
                for (int col = max(64 * h, r); col < 64 * h + 64; ++col) u = fmaf(cur[r * SLD + col], tv[col], u);
                red[h * QB + r] = u;
                __syncthreads();
                if (tid < QB) b[(int64_t)i * QB + tid] = red[tid] + red[QB + tid];
            }
            __syncthreads();
        }
    }
}

// block sum (deterministic), result in every thread
__device__ double tc_block_sum(TcCtx &c, double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) c.red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < QTHREADS / 32; ++w) s += c.red[w];
    __syncthreads();
    return s;
}

__device__ bool tc_solve(TcCtx &c, const DagProb &P) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * QB;
    double *r = P.vec, *al = P.vec + m, *tt = P.vec + 3 * m;
    if (!dag_failed(P)) {
        for (int i = 0; i < T; ++i)
            for (int j = 0; j <= i; ++j)
                if (!dag_wait(f_L(P) + tile_index(T, i, j), 1, c.h, P.info, c.ok)) return false;
        double rr = 0.0;
        for (int64_t e = tid; e < m; e += QTHREADS) {
            const double v = e < P.n ? P.y[e] - (P.mu ? P.mu[e] : 0.0) : 0.0;
            if (!isfinite(v)) set_info(P.info, -2);
            r[e] = v;
            al[e] = v;
            rr = fma(v, v, rr);
        }
        const double rn = tc_block_sum(c, rr);
        if (tid == 0) P.part[T + 3 * dag_ntiles(T) + 1] = rn;  // ||r||^2
        __syncthreads();
        lowp_solve(c, P, al, tt);
    }
    dag_signal(f_solved(P));
    return true;
}

// Residual partials of one lower tile (i, j) for evaluation e: with the
// tile's entries C_ij in double-float (evaluated once),
//   rp[t][0][r] = sum_c C_ij(r, c) alpha_j(c),   rp[t][1][c] = sum_r C_ij(r, c) alpha_i(r)
// (the second for i > j only: C is symmetric).  Rows and columns beyond n
// contribute nothing.
__device__ bool tc_res(TcCtx &c, const DagProb &P, int e, int i, int j) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * QB;
    const double *al = P.vec + m;
    int *wait_f = e == 0 ? f_solved(P) : f_corr(P, e - 1);
    if (!dag_wait(wait_f, 1, c.h, P.info, c.ok)) return false;
    const bool skip = dag_uniform(failed(P.info) || *reinterpret_cast<volatile int *>(f_conv(P)));
    if (threadIdx.x == 0) c.misc[1] = skip ? 1 : 0;
    if (!skip) {
        float2 *stg = reinterpret_cast<float2 *>(c.opA);
        float2 *avr = reinterpret_cast<float2 *>(c.opA + 2 * QOPER - 4096);  // alpha of the rows
        float2 *pr = reinterpret_cast<float2 *>(c.red);                      // [2][128]
        __syncthreads();
        if (tid < QB) {
            const int64_t gc = (int64_t)j * QB + tid, gr = (int64_t)i * QB + tid;
            c.xs[tid] = df_point(gc < P.n ? P.x[gc] : make_double2(0.0, 0.0));
            const dfl ac = d2df(gc < P.n ? __ldcg(al + gc) : 0.0);
            c.av[tid] = make_float2(ac.h, ac.l);
            const dfl ar = d2df(gr < P.n ? __ldcg(al + gr) : 0.0);
            avr[tid] = make_float2(ar.h, ar.l);
        }
        __syncthreads();
        const int r = tid & (QB - 1), h = tid >> 7;
        const int64_t gi = (int64_t)i * QB + r;
        const bool row_ok = gi < P.n;
        const float4 xi = df_point(row_ok ? P.x[gi] : make_double2(0.0, 0.0));
        // rows: four independent chains (columns mod 4)
        dfl a0{0.0f, 0.0f}, a1{0.0f, 0.0f}, a2{0.0f, 0.0f}, a3{0.0f, 0.0f};
        for (int col = 64 * h; col < 64 * h + 64; col += 4) {
            dfl v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t gc = (int64_t)j * QB + col + u;
                dfl cv, unused;
                df_cov_s<false>(P.kind, P.dscale, P.ds2, df_dist(xi, c.xs[col + u]), c.tab, cv,
                                unused);
                const bool in = row_ok && gc < P.n;
                v[u] = !in ? dfl{0.0f, 0.0f} : (gc == gi ? P.ddiag : cv);
                stg[r * QSTG_LD + col + u] = make_float2(v[u].h, v[u].l);
            }
            a0 = df_add(a0, df_mul(v[0], dfl{c.av[col].x, c.av[col].y}));
            a1 = df_add(a1, df_mul(v[1], dfl{c.av[col + 1].x, c.av[col + 1].y}));
            a2 = df_add(a2, df_mul(v[2], dfl{c.av[col + 2].x, c.av[col + 2].y}));
            a3 = df_add(a3, df_mul(v[3], dfl{c.av[col + 3].x, c.av[col + 3].y}));
        }
        a0 = df_add(a0, a2);
        a1 = df_add(a1, a3);
        const dfl a = df_add(a0, a1);
        pr[h * QB + r] = make_float2(a.h, a.l);
        __syncthreads();
        double *rp = P.rp + (size_t)tile_index(T, i, j) * (2 * QB);
        if (tid < QB) {
            const dfl t = df_add(dfl{pr[tid].x, pr[tid].y}, dfl{pr[QB + tid].x, pr[QB + tid].y});
            rp[tid] = df_to_double(t);
        }
        if (i != j) {
            // columns: thread (column r, rows 64h..)
            __syncthreads();
            dfl b0{0.0f, 0.0f}, b1{0.0f, 0.0f};
            for (int row = 64 * h; row < 64 * h + 64; row += 2) {
                const float2 v0 = stg[row * QSTG_LD + r], v1 = stg[(row + 1) * QSTG_LD + r];
                b0 = df_add(b0, df_mul(dfl{v0.x, v0.y}, dfl{avr[row].x, avr[row].y}));
                b1 = df_add(b1, df_mul(dfl{v1.x, v1.y}, dfl{avr[row + 1].x, avr[row + 1].y}));
            }
            const dfl b = df_add(b0, b1);
            __syncthreads();
            pr[h * QB + r] = make_float2(b.h, b.l);
            __syncthreads();
            if (tid < QB) {
                const dfl t = df_add(dfl{pr[tid].x, pr[tid].y}, dfl{pr[QB + tid].x, pr[QB + tid].y});
                rp[QB + tid] = df_to_double(t);
            }
        }
    }
    dag_signal(f_res(P, e));
    return true;
}

// s = r - C alpha from the tile partials (fixed order: deterministic),
// ||s|| / ||r|| returned to every thread.
__device__ double tc_combine(TcCtx &c, const DagProb &P) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * QB;
    const double *r = P.vec;
    double *s = P.vec + 2 * m;
    double sq = 0.0;
    for (int64_t g = tid; g < m; g += QTHREADS) {
        const int I = (int)(g / QB), rr = (int)(g % QB);
        double acc = 0.0;
        if (g < P.n) {
            for (int jj = 0; jj <= I; ++jj) acc += __ldcg(P.rp + (size_t)tile_index(T, I, jj) * (2 * QB) + rr);
            for (int ii = I + 1; ii < T; ++ii)
                acc += __ldcg(P.rp + (size_t)tile_index(T, ii, I) * (2 * QB) + QB + rr);
        }
        const double sv = g < P.n ? __ldcg(r + g) - acc : 0.0;
        s[g] = sv;
        sq = fma(sv, sv, sq);
    }
    const double tot = tc_block_sum(c, sq);
    const double rn = __ldcg(P.part + T + 3 * dag_ntiles(T) + 1);
    return rn > 0.0 ? sqrt(tot / rn) : 0.0;
}

__device__ bool tc_corr(TcCtx &c, const DagProb &P, int e) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * QB;
    if (!dag_wait(f_res(P, e), dag_ntiles(T), c.h, P.info, c.ok)) return false;
    int *conv = f_conv(P);
    if (!dag_uniform(failed(P.info) || *reinterpret_cast<volatile int *>(conv))) {
        const double ratio = tc_combine(c, P);
        double *stat = P.part + T + 3 * dag_ntiles(T);
        if (ratio <= QREFINE_TOL) {
            if (tid == 0) {
                *stat = ratio;
                *conv = 1;
            }
        } else {
            double *al = P.vec + m, *s = P.vec + 2 * m, *tt = P.vec + 3 * m;
            __syncthreads();
            lowp_solve(c, P, s, tt);
            for (int64_t q = tid; q < m; q += QTHREADS) al[q] += s[q];
        }
    }
    dag_signal(f_corr(P, e));
    return true;
}

__device__ bool tc_finll(TcCtx &c, const DagProb &P) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * QB;
    if (!dag_wait(f_res(P, DAG_EVALS - 1), dag_ntiles(T), c.h, P.info, c.ok)) return false;
    if (!dag_failed(P)) {
        double *stat = P.part + T + 3 * dag_ntiles(T);
        const bool conv = dag_uniform(*reinterpret_cast<volatile int *>(f_conv(P)) != 0);
        const double ratio = conv ? __ldcg(stat) : tc_combine(c, P);
        const double *r = P.vec, *al = P.vec + m;
        double q = 0.0;
        for (int64_t e = tid; e < P.n; e += QTHREADS) q = fma(__ldcg(r + e), __ldcg(al + e), q);
        const double quad = tc_block_sum(c, q);
        if (tid == 0) {
            double ld = 0.0;
            for (int i = 0; i < T; ++i) ld += __ldcg(P.part + i);
            const double logdet = 2.0 * ld;
            const double LOG_2PI = 1.8378770664093454836;
            const bool bad = failed(P.info);
            P.out[0] = bad ? nan("") : -0.5 * logdet - 0.5 * quad - 0.5 * (double)P.n * LOG_2PI;
            P.out[1] = bad ? nan("") : logdet;
            P.out[2] = bad ? nan("") : quad;
            P.out[3] = bad ? nan("") : ratio;
        }
    } else if (tid == 0) {
        P.out[0] = P.out[1] = P.out[2] = P.out[3] = nan("");
    }
    dag_signal(f_fin(P));
    return true;
}

__device__ bool tc_lg(TcCtx &c, const DagProb &P, int i, int j) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * QB;
    int *Xf = f_X(P);
    double g0 = 0.0, g2 = 0.0;
    dfl h0{0.0f, 0.0f}, h1{0.0f, 0.0f};
    if (!dag_failed(P)) {
        auto pair = [&](int q, const uint8_t *&ga, const uint8_t *&gb) -> bool {
            const int mm = i + q;
            if (!dag_wait(Xf + tile_index(T, mm, i), 1, c.h, P.info, c.ok)) return false;
            if (!dag_wait(Xf + tile_index(T, mm, j), 1, c.h, P.info, c.ok)) return false;
            ga = store_tile(P.XSc, T, mm, i);
            gb = store_tile(P.XSc, T, mm, j);
            return true;
        };
        if (!tc_contract(c, P, T - i, pair)) return false;
        if (!dag_wait(f_fin(P), 1, c.h, P.info, c.ok)) return false;
        const double *al = P.vec + m;
        __syncthreads();
        stage_points(c, P, j);
        if (tid < QB) {
            const dfl a = d2df(__ldcg(al + (int64_t)j * QB + tid));
            c.av[tid] = make_float2(a.h, a.l);
        }
        __syncthreads();
        const int w = tid >> 5, lane = tid & 31, qd = w & 3, ch = w >> 2;
        const int row = qd * 32 + lane;
        const int64_t gi = (int64_t)i * QB + row;
        const bool row_ok = gi < P.n;
        const float4 xi = df_point(row_ok ? P.x[gi] : make_double2(0.0, 0.0));
        const double ai = row_ok ? __ldcg(al + gi) : 0.0;
        const dfl aid = d2df(ai);
        dfl h2{0.0f, 0.0f}, h3{0.0f, 0.0f};
        for (int g = 0; g < 4; ++g) {
            dfl wv[16];
            run_ld16(c, ch * 64 + g * 16, wv);  // every lane: tcgen05.ld is warp-collective
#pragma unroll 4
            for (int jj = 0; jj < 16; ++jj) {
                const int col = ch * 64 + g * 16 + jj;
                const int64_t gc = (int64_t)j * QB + col;
                dfl cv, dr;
                df_cov_s<true>(P.kind, P.dscale, P.ds2, df_dist(xi, c.xs[col]), c.tab, cv, dr);
                const bool off = row_ok && gc < gi && gc < P.n;
                if (row_ok && gc == gi) {
                    const double cb = 0.5 * (ai * ai - df_to_double(wv[jj]));
                    g0 = fma(cb, P.s2, g0);
                    g2 = fma(cb, P.tau2, g2);
                }
                const dfl cb2 = df_add(df_mul(aid, dfl{c.av[col].x, c.av[col].y}), df_neg(wv[jj]));
                const dfl t0 = off ? df_mul(cb2, cv) : dfl{0.0f, 0.0f};
                const dfl t1 = off ? df_mul(cb2, dr) : dfl{0.0f, 0.0f};
                if (jj & 1) {
                    h2 = df_add(h2, t0);
                    h3 = df_add(h3, t1);
                } else {
                    h0 = df_add(h0, t0);
                    h1 = df_add(h1, t1);
                }
            }
        }
        h0 = df_add(h0, h2);
        h1 = df_add(h1, h3);
    }
    g0 += df_to_double(h0);
    double g1 = df_to_double(h1);
    for (int o = 16; o > 0; o >>= 1) {
        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
        g1 += __shfl_xor_sync(0xffffffffu, g1, o);
        g2 += __shfl_xor_sync(0xffffffffu, g2, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) {
        c.red[tid >> 5] = g0;
        c.red[8 + (tid >> 5)] = g1;
        c.red[16 + (tid >> 5)] = g2;
    }
    __syncthreads();
    if (tid < 3) {
        double s = 0.0;
        for (int w8 = 0; w8 < QTHREADS / 32; ++w8) s += c.red[8 * tid + w8];
        P.part[T + 3 * tile_index(T, i, j) + tid] = s;
    }
    dag_signal(f_lg(P));
    return true;
}

__device__ bool tc_final(TcCtx &c, const DagProb &P) {
    const int T = P.T, tid = threadIdx.x;
    const int nt = dag_ntiles(T);
    if (!dag_wait(f_lg(P), nt, c.h, P.info, c.ok)) return false;
    const bool bad = dag_failed(P);
    double s[3] = {0.0, 0.0, 0.0}, cc[3] = {0.0, 0.0, 0.0};
    for (int t = tid; t < nt; t += QTHREADS)
        for (int q = 0; q < 3; ++q) {
            const double x = __ldcg(P.part + T + 3 * t + q), u = s[q] + x;
            cc[q] += (fabs(s[q]) >= fabs(x)) ? (s[q] - u) + x : (x - u) + s[q];
            s[q] = u;
        }
    double *buf = reinterpret_cast<double *>(c.opB);  // [3][256]
    __syncthreads();
    for (int q = 0; q < 3; ++q) buf[q * QTHREADS + tid] = s[q] + cc[q];
    __syncthreads();
    if (tid < 3) {
        double S = 0.0, C = 0.0;
        for (int t = 0; t < QTHREADS; ++t) {
            const double x = buf[tid * QTHREADS + t], u = S + x;
            C += (fabs(S) >= fabs(x)) ? (S - u) + x : (x - u) + S;
            S = u;
        }
        P.grad[tid] = bad ? nan("") : S + C;
    }
    dag_signal(P.flag + dag_done_flag(T, 1));
    __syncthreads();
    return true;
}

__global__ void __launch_bounds__(QTHREADS, 1)
    dag_tc_kernel(DagHdr *h, const DagProb *probs, const int2 *list, int ntot, const double *tab,
                  const float2 *dftab, double *scratch) {
    extern __shared__ uint8_t q_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(q_smem_raw) + 1023) &
                                              ~static_cast<uintptr_t>(1023));
    TcCtx c;
    c.opA = sm + QS_OPA;
    c.opB = sm + QS_OPB;
    c.exA = reinterpret_cast<int *>(sm + QS_EXA);
    c.exB = reinterpret_cast<int *>(sm + QS_EXB);
    c.tab = reinterpret_cast<float2 *>(sm + QS_TAB);
    c.xs = reinterpret_cast<float4 *>(sm + QS_X);
    c.av = reinterpret_cast<float2 *>(sm + QS_AV);
    c.red = reinterpret_cast<double *>(sm + QS_RED);
    c.emax = reinterpret_cast<float *>(sm + QS_EMAX);
    c.mbar = reinterpret_cast<uint64_t *>(sm + QS_MISC);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + QS_MISC + 8);
    c.ok = reinterpret_cast<int *>(sm + QS_MISC + 16);
    c.misc = reinterpret_cast<int *>(sm + QS_MISC + 32);
    c.phase = 0;
    c.h = h;
    c.scr = scratch + (size_t)blockIdx.x * QSCRATCH_DOUBLES;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int q = tid; q < DF_TAB; q += QTHREADS) c.tab[q] = dftab[q];
    if (tid == 0) {
        mbar_init(c.mbar, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    c.tmem = *tslot;
    for (;;) {
        if (tid == 0) c.misc[0] = ld_relaxed_gpu(&h->abort) ? ntot : atomicAdd(&h->next, 1);
        __syncthreads();
        const int t = c.misc[0];
        __syncthreads();
        if (t >= ntot) break;
        const int2 e = list[t];
        const DagProb &P = probs[e.x];
        int i = 0, k = 0;
        const int type = dag_decode(P.T, P.mixed, e.y, i, k);
        if (!P.mixed) {
            // a problem on FP64 tiles: the FP64 tasks, their shared memory
            // laid over the operand buffers
            DagSmem &dsm = *reinterpret_cast<DagSmem *>(c.opA);
            __syncthreads();
            if (tid < EXP_TAB) dsm.tab[tid] = tab[tid];
            __syncthreads();
            const long long c0 = dag_stat_begin(h, dsm.ok);
            bool ok = true;
            switch (type) {
                case DT_CHOL: ok = task_chol(P, i, k, dsm, h); break;
                case DT_SOLVE: ok = task_solve(P, dsm, h); break;
                case DT_TRTRI: ok = task_trtri(P, i, k, dsm, h); break;
                case DT_LG: ok = task_lg(P, i, k, dsm, h); break;
                default: ok = task_final(P, dsm, h); break;
            }
            dag_stat_end(h, (type == DT_CHOL && i == k) ? 8 : type, c0, dsm.ok);
            if (!ok) break;
            continue;
        }
        const long long c0 = dag_stat_begin(h, c.ok);
        bool ok = true;
        switch (type) {
            case DT_CHOL: ok = tc_chol(c, P, i, k); break;
            case DT_SOLVE: ok = tc_solve(c, P); break;
            case DT_TRTRI: ok = tc_trtri(c, P, i, k); break;
            case DT_RES:
                c.misc[1] = 0;
                ok = tc_res(c, P, k, i & 0xffff, i >> 16);
                break;
            case DT_CORR: ok = tc_corr(c, P, k); break;
            case DT_FINLL: ok = tc_finll(c, P); break;
            case DT_LG: ok = tc_lg(c, P, i, k); break;
            default: ok = tc_final(c, P); break;
        }
        // class 9: a residual task of a problem already converged (no work)
        const int cls = (type == DT_CHOL && i == k) ? 8 : (type == DT_RES && c.misc[1]) ? 9 : type;
        dag_stat_end(h, cls, c0, c.ok);
        if (!ok) break;
    }
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(c.tmem, 512);
    }
}

int dag_tc_launch(int grid, DagHdr *hdr, const DagProb *probs, const int2 *list, int ntot,
                  const double *tab, const float2 *dftab, double *scratch, cudaStream_t s) {
    // set once per device; a race between host threads only repeats the
    // (idempotent) attribute call
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
    if (!attr_set[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(dag_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 QS_DYN) != cudaSuccess)
            return GP_ERR_CUDA;
        attr_set[dev].store(true, std::memory_order_release);
    }
    dag_tc_kernel<<<grid, QTHREADS, QS_DYN, s>>>(hdr, probs, list, ntot, tab, dftab, scratch);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

}  // namespace gp
