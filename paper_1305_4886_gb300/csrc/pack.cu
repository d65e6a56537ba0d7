// pack.cu -- FP64 operands into 16-bit slice stores for the tensor-core
// contractions (the row-scaled splits of the mixed and FP64-grade forms).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "kern_df.cuh"
#include "tc_gemm.h"

namespace gp {

// ---------------------------------------------------------------------------
// Row-scaled split of FP64 operands into three BF16 slices (see the top of
// this file).  The operand element (r, k) is
//   trans = 0: src[r + k ld]   (operand rows are rows of the column-major
//                               source, K runs along its columns)
//   trans = 1: src[k + r ld]   (operand rows are source columns)
// lower_mask: entries above the source diagonal are treated as zero
// (trans = 0: r + diag_off < k; trans = 1: k + diag_off < r), for triangular
// sources whose upper part holds stale data.  One CTA packs 32 rows over a
// 512-column chunk of K: pass 1 finds each row's bound 2^e_r over the chunk
// (so the leading products are exact within every 512-deep chunk of a
// contraction whose operands share the chunking), pass 2 writes the
// slices with k contiguous (trans = 0 goes through a shared-memory
// transpose so that both the FP64 reads and the BF16 writes are coalesced).
// The split runs in FP32 after one FP64 -> (hi, lo) FP32 conversion.
// ---------------------------------------------------------------------------
struct SplitArgs {
    const double *src;
    int64_t ld, R, K, Kvalid;
    int trans;
    int64_t diag_off;
    int lower_mask;
    int S;      // 3: normalized FP16 slices + row exponents; 5: scaled BF16 integer slices
    uint16_t *dst;
    int *dst_ex;
    int64_t ex_ld;
    int64_t dst_rows, dst_kld, dst_row_off, dst_k_off;
    int64_t kch;  // K chunk of one CTA and of one row bound
};

// raw bits of operand element (r, k); masked and out-of-range entries are +0
__device__ __forceinline__ unsigned long long split_get(const SplitArgs &a, int64_t r, int64_t k) {
    if (r >= a.R || k >= a.Kvalid) return 0ull;
    if (a.lower_mask) {
        if (a.trans ? (k + a.diag_off < r) : (r + a.diag_off < k)) return 0ull;
    }
    const double v = a.trans ? a.src[k + r * a.ld] : a.src[r + k * a.ld];
    return static_cast<unsigned long long>(__double_as_longlong(v));
}

// Normalized slices of one entry (mixed form), given the row's scale
// sc = 2^{7-e}: with y = x sc held as a double-float (exact scaling),
// s0 = round(y) (an integer in [-128, 128]), s1 = fp16(y - s0),
// s2 = fp16(y - s0 - s1); y is then carried to about 2^-25 (2^{e-32} of x).
__device__ __forceinline__ void split3_norm(unsigned long long u, float sc, uint16_t (&s)[3]) {
    const dfl x = f64_to_df(u);
    const float yh = x.h * sc, yl = x.l * sc;
    const float q = rintf(yh);
    float t, e;
    {
        const dfl te = df_two_sum(__fsub_rn(yh, q), yl);  // yh - q is exact
        t = te.h;
        e = te.l;
    }
    const __half h1 = __float2half_rn(t);
    const float rest = __fadd_rn(__fsub_rn(t, __half2float(h1)), e);  // t - h1 exact
    s[0] = __half_as_ushort(__float2half_rn(q));
    s[1] = __half_as_ushort(h1);
    s[2] = __half_as_ushort(__float2half_rn(rest));
}

// Integer slices on the row grid (FP64-grade mode): with y = x 2^{7-e} held
// as a double-float, q_p = round(y_p), y_{p+1} = 256 (y_p - q_p); slice p is
// q_p 2^{e-7-8p} (|q_p| <= 256, exact in BF16).  Five slices carry x to
// 2^{e-40}.  All products of slice group d = p + q are then integers times
// one power of two per output entry, so the leading groups accumulate
// exactly in FP32 (see the top of this file for the depth limits).
__device__ __forceinline__ void split_ozaki(unsigned long long u, float sc, float isc,
                                            uint16_t (&s)[5]) {
    const dfl x = f64_to_df(u);
    float yh = x.h * sc, yl = x.l * sc, w = isc;
#pragma unroll
    for (int p = 0; p < 5; ++p) {
        const float q = rintf(yh);
        s[p] = __bfloat16_as_ushort(__float2bfloat16_rn(q * w));
        float h, l;
        const float d = __fsub_rn(yh, q);  // exact
        const float t = __fadd_rn(d, yl);
        const float bb = __fsub_rn(t, d);
        l = __fadd_rn(__fsub_rn(d, __fsub_rn(t, bb)), __fsub_rn(yl, bb));
        h = t;
        yh = h * 256.0f;
        yl = l * 256.0f;
        w *= (1.0f / 256.0f);
    }
}

constexpr int64_t SPLIT_KCH = TC_CHUNK_K;  // K chunk of one CTA (and of one row bound)
constexpr int SPLIT_MAX_S = 5;

__global__ void __launch_bounds__(256) split_rows_kernel(SplitArgs a) {
    __shared__ unsigned long long pmax[8][32];
    __shared__ float sc_s[32], isc_s[32];
    __shared__ unsigned short tile[SPLIT_MAX_S][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    // this CTA's K chunk; each (row, chunk) gets its own bound 2^e
    const int64_t kb = (int64_t)blockIdx.y * a.kch;
    const int64_t ke = min(a.K, kb + a.kch);
    const int64_t kev = min(ke, a.Kvalid);
    constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
    // pass 1: row bounds, as the largest magnitude's bit pattern
    if (a.trans == 0) {
        unsigned long long m = 0ull;
        for (int64_t k = kb + warp; k < kev; k += 8) {
            const unsigned long long v = split_get(a, r0 + lane, k) & ABS;
            m = v > m ? v : m;
        }
        pmax[warp][lane] = m;
    } else {
        for (int i = warp; i < 32; i += 8) {
            unsigned long long m = 0ull;
            for (int64_t k = kb + lane; k < kev; k += 32) {
                const unsigned long long v = split_get(a, r0 + i, k) & ABS;
                m = v > m ? v : m;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
                m = t > m ? t : m;
            }
            if (lane == 0) {
                pmax[0][i] = m;
                for (int w = 1; w < 8; ++w) pmax[w][i] = 0ull;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long m = 0ull;
        for (int w = 0; w < 8; ++w) m = pmax[w][threadIdx.x] > m ? pmax[w][threadIdx.x] : m;
        // every entry of the row is below 2^e, e = unbiased exponent of the max + 1
        int e = 0;
        const int E = static_cast<int>(m >> 52);
        if (E > 0) e = E - 1022;
        e = max(-100, min(e, 120));
        sc_s[threadIdx.x] = ldexpf(1.0f, 7 - e);
        isc_s[threadIdx.x] = ldexpf(1.0f, e - 7);
        if (a.dst_ex && r0 + threadIdx.x < a.R)
            a.dst_ex[(a.dst_row_off + r0 + threadIdx.x) * a.ex_ld + (a.dst_k_off + kb) / a.kch] = e;
    }
    __syncthreads();
    const int64_t slice = a.dst_rows * a.dst_kld;
    uint16_t *d0 = a.dst + (a.dst_row_off + r0) * a.dst_kld + a.dst_k_off;
    if (a.trans == 0) {
        for (int64_t kc = kb; kc < ke; kc += 32) {
            // lane = row: coalesced FP64 reads down each column
            for (int i = warp; i < 32; i += 8) {
                uint16_t s[SPLIT_MAX_S] = {0, 0, 0, 0, 0};
                const unsigned long long u = split_get(a, r0 + lane, kc + i);
                if (a.S == 5) {
                    split_ozaki(u, sc_s[lane], isc_s[lane], s);
                } else {
                    uint16_t t3[3];
                    split3_norm(u, sc_s[lane], t3);
                    s[0] = t3[0];
                    s[1] = t3[1];
                    s[2] = t3[2];
                }
#pragma unroll
                for (int p = 0; p < SPLIT_MAX_S; ++p) tile[p][i][lane] = s[p];
            }
            __syncthreads();
            // lane = k: coalesced BF16 writes along each row
            for (int i = warp; i < 32; i += 8) {
                const int64_t r = r0 + i, k = kc + lane;
                if (r < a.R && k < ke) {
                    for (int p = 0; p < a.S; ++p)
                        d0[p * slice + (int64_t)i * a.dst_kld + k] = tile[p][lane][i];
                }
            }
            __syncthreads();
        }
    } else {
        for (int i = warp; i < 32; i += 8) {
            const int64_t r = r0 + i;
            if (r >= a.R) continue;
            for (int64_t k = kb + lane; k < ke; k += 32) {
                uint16_t s[SPLIT_MAX_S] = {0, 0, 0, 0, 0};
                const unsigned long long u = split_get(a, r, k);
                if (a.S == 5) {
                    split_ozaki(u, sc_s[i], isc_s[i], s);
                } else {
                    uint16_t t3[3];
                    split3_norm(u, sc_s[i], t3);
                    s[0] = t3[0];
                    s[1] = t3[1];
                    s[2] = t3[2];
                }
                for (int p = 0; p < a.S; ++p) d0[p * slice + (int64_t)i * a.dst_kld + k] = s[p];
            }
        }
    }
}

// The three-slice split with vector memory access (the mixed form's hot
// case): the same row bounds and slices as split_rows_kernel, one CTA per 32
// rows x one 512-deep K chunk.  trans = 1 (operand rows contiguous in K):
// split3_vec_kernel, double2 loads along K and 8-byte slice stores.
// trans = 0 (operand rows are rows of the column-major source):
// split3_panel_kernel, double2 loads down the columns, the slices transposed
// through shared memory in 64-column steps and stored 16 bytes per thread.
// Both require K % 64 == 0, a 16-byte aligned source and an even ld.
__device__ __forceinline__ unsigned long long split_bits(const SplitArgs &a, int64_t r, int64_t k,
                                                         double v) {
    if (r >= a.R || k >= a.Kvalid) return 0ull;
    if (a.lower_mask && (a.trans ? (k + a.diag_off < r) : (r + a.diag_off < k))) return 0ull;
    return static_cast<unsigned long long>(__double_as_longlong(v));
}

// two consecutive operand entries along the source's contiguous direction
__device__ __forceinline__ void split_pair(const SplitArgs &a, int64_t r, int64_t k, bool along_k,
                                           unsigned long long &u0, unsigned long long &u1) {
    // along_k: (r, k), (r, k + 1) at src[k + r ld]; else (r, k), (r + 1, k) at src[r + k ld]
    const int64_t r1 = along_k ? r : r + 1, k1 = along_k ? k + 1 : k;
    const double *p = along_k ? a.src + k + r * a.ld : a.src + r + k * a.ld;
    if (r1 < a.R && k1 < a.Kvalid && r < a.R && k < a.Kvalid) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        u0 = split_bits(a, r, k, v.x);
        u1 = split_bits(a, r1, k1, v.y);
    } else {
        u0 = (r < a.R && k < a.Kvalid) ? split_bits(a, r, k, p[0]) : 0ull;
        u1 = (r1 < a.R && k1 < a.Kvalid) ? split_bits(a, r1, k1, p[along_k ? 1 : 1]) : 0ull;
    }
}

constexpr int SPV_LD = 72;  // shared row stride of the transpose tile (16-byte rows)

// trans = 1 only (trans = 0 is split3_panel_kernel)
__global__ void __launch_bounds__(256) split3_vec_kernel(SplitArgs a) {
    __shared__ unsigned long long pm[32];
    __shared__ float sc_s[32];
    constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int64_t kb = (int64_t)blockIdx.y * a.kch;
    const int64_t ke = min(a.K, kb + a.kch);
    const int64_t slice = a.dst_rows * a.dst_kld;
    uint16_t *d0 = a.dst + (a.dst_row_off + r0) * a.dst_kld + a.dst_k_off;
    // warp: rows r0 + warp + 8i; lane: K quads kb + 4 lane + 128 j
    unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
    for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + warp + 8 * i;
        for (int64_t k = kb + 4 * lane; k < ke; k += 128) {
            unsigned long long u[4];
            split_pair(a, r, k, true, u[0], u[1]);
            split_pair(a, r, k + 2, true, u[2], u[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q) m[i] = max(m[i], u[q] & ABS);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[i] = max(m[i], __shfl_xor_sync(0xffffffffu, m[i], o));
        if (lane == 0) pm[warp + 8 * i] = m[i];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned long long m = pm[threadIdx.x];
        int e = 0;
        const int E = static_cast<int>(m >> 52);
        if (E > 0) e = E - 1022;
        e = max(-100, min(e, 120));
        sc_s[threadIdx.x] = ldexpf(1.0f, 7 - e);
        if (r0 + threadIdx.x < a.R)
            a.dst_ex[(a.dst_row_off + r0 + threadIdx.x) * a.ex_ld + (a.dst_k_off + kb) / a.kch] = e;
    }
    __syncthreads();
    for (int i = 0; i < 4; ++i) {
        const int rl = warp + 8 * i;
        const int64_t r = r0 + rl;
        if (r >= a.R) continue;
        const float sc = sc_s[rl];
        for (int64_t k = kb + 4 * lane; k < ke; k += 128) {
            unsigned long long u[4];
            split_pair(a, r, k, true, u[0], u[1]);
            split_pair(a, r, k + 2, true, u[2], u[3]);
            uint16_t t[4][3];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint16_t s3[3];
                split3_norm(u[q], sc, s3);
                t[q][0] = s3[0];
                t[q][1] = s3[1];
                t[q][2] = s3[2];
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                uint2 v;
                v.x = t[0][p] | ((uint32_t)t[1][p] << 16);
                v.y = t[2][p] | ((uint32_t)t[3][p] << 16);
                *reinterpret_cast<uint2 *>(d0 + p * slice + (int64_t)rl * a.dst_kld + (k - kb) + kb) = v;
            }
        }
    }
}

// The trans = 0 case in one pass over the source: each thread keeps its 16
// entry pairs in registers between the row-bound reduction and the split,
// where the two-pass form read the panel twice (the second time often from
// DRAM again) and waited on each 64-column step's loads in turn.  One CTA of
// 256 R threads covers 16 rows x one 512 R-deep chunk (R = 1, or 2 for the
// three-slice stores bounded over 1024 columns); with R = 1 two CTAs share
// an SM, so that one's loads overlap the other's split and stores.  Same
// bounds, slices and layout.
constexpr int SPP_ROWS = 16;

template <int R>
__global__ void __launch_bounds__(256 * R, 2 / R) split3_panel_kernel(SplitArgs a) {
    constexpr int NT = 256 * R;       // threads
    constexpr int KCH = 512 * R;      // chunk (and row bound) width
    constexpr int CS = 32 * R;        // column stride of a thread's pairs
    constexpr int PPS = 2 / R;        // a thread's pairs per 64-column step
    __shared__ unsigned long long pm[NT / 32][SPP_ROWS];
    __shared__ float sc_s[SPP_ROWS];
    __shared__ __align__(16) uint16_t tile[2][3][SPP_ROWS][SPV_LD];
    constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * SPP_ROWS;
    const int64_t kb = (int64_t)blockIdx.y * KCH;
    const int64_t ke = min(a.K, kb + KCH);
    const int64_t slice = a.dst_rows * a.dst_kld;
    uint16_t *d0 = a.dst + (a.dst_row_off + r0) * a.dst_kld + a.dst_k_off;
    // lane: rows rp and rp + 1; columns kb + kc + CS i (i < 16), kc = 4 warp + (lane / 8)
    const int rp = 2 * (lane & 7), kc = 4 * warp + (lane >> 3);
    unsigned long long u[16][2];
    unsigned long long m0 = 0ull, m1 = 0ull;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int64_t k = kb + kc + CS * i;
        if (k < ke) {
            split_pair(a, r0 + rp, k, false, u[i][0], u[i][1]);
        } else {
            u[i][0] = u[i][1] = 0ull;
        }
        m0 = max(m0, u[i][0] & ABS);
        m1 = max(m1, u[i][1] & ABS);
    }
    // lanes l, l + 8, l + 16, l + 24 hold the same rows
    m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, 8));
    m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, 8));
    m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, 16));
    m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, 16));
    if (lane < 8) {
        pm[warp][rp] = m0;
        pm[warp][rp + 1] = m1;
    }
    __syncthreads();
    if (threadIdx.x < SPP_ROWS) {
        unsigned long long m = 0ull;
        for (int w = 0; w < NT / 32; ++w) m = max(m, pm[w][threadIdx.x]);
        int e = 0;
        const int E = static_cast<int>(m >> 52);
        if (E > 0) e = E - 1022;
        e = max(-100, min(e, 120));
        sc_s[threadIdx.x] = ldexpf(1.0f, 7 - e);
        if (r0 + threadIdx.x < a.R)
            a.dst_ex[(a.dst_row_off + r0 + threadIdx.x) * a.ex_ld + (a.dst_k_off + kb) / KCH] = e;
    }
    __syncthreads();
    const float sc0 = sc_s[rp], sc1 = sc_s[rp + 1];
    // 64-column steps: this thread's pairs PPS c + h (h < PPS) lie in step c,
    // at its columns kc + CS h; the transpose tile is double-buffered (one
    // barrier per step: a buffer is rewritten only after the barrier that
    // follows its stores)
#pragma unroll
    for (int c = 0; c < KCH / 64; ++c) {
        if (kb + 64 * c >= ke) break;  // uniform
        uint16_t(*t)[SPP_ROWS][SPV_LD] = tile[c & 1];
#pragma unroll
        for (int h = 0; h < PPS; ++h) {
            const int kk = kc + CS * h;
            uint16_t s3[3];
            split3_norm(u[PPS * c + h][0], sc0, s3);
            t[0][rp][kk] = s3[0];
            t[1][rp][kk] = s3[1];
            t[2][rp][kk] = s3[2];
            split3_norm(u[PPS * c + h][1], sc1, s3);
            t[0][rp + 1][kk] = s3[0];
            t[1][rp + 1][kk] = s3[1];
            t[2][rp + 1][kk] = s3[2];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < 3 * SPP_ROWS * 8; idx += NT) {
            const int p = idx / (SPP_ROWS * 8), row = (idx >> 3) % SPP_ROWS, ch = idx & 7;
            if (r0 + row < a.R)
                *reinterpret_cast<uint4 *>(d0 + p * slice + (int64_t)row * a.dst_kld + kb + 64 * c + 8 * ch) =
                    *reinterpret_cast<const uint4 *>(&t[p][row][8 * ch]);
        }
    }
}

int split_rows(const double *src, int64_t ld, int64_t R, int64_t K, int64_t Kvalid, int trans,
               int64_t diag_off, int lower_mask, int S, uint16_t *dst, int *dst_ex,
               int64_t dst_rows, int64_t dst_kld, int64_t dst_row_off, int64_t dst_k_off,
               cudaStream_t s, int64_t kch) {
    if (R <= 0 || K <= 0) return GP_OK;
    if ((S != 3 && S != 5) || (S == 3) != (dst_ex != nullptr) || dst_row_off + R > dst_rows ||
        dst_k_off + K > dst_kld || !(kch == SPLIT_KCH || (kch == 2 * SPLIT_KCH && S == 3)) ||
        dst_k_off % kch)
        return GP_ERR_INVALID;
    SplitArgs a{src, ld, R, K, Kvalid < K ? Kvalid : K, trans, diag_off, lower_mask, S,
                dst, dst_ex, tc_ex_ld(dst_kld, kch), dst_rows, dst_kld, dst_row_off, dst_k_off,
                kch};
    const int ev = prof_start(s);
    dim3 g((unsigned)ceil_div(R, 32), (unsigned)ceil_div(K, kch));
    const bool vec = S == 3 && K % 64 == 0 && ld % 2 == 0 &&
                     reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(dst) % 16 == 0 && dst_kld % 64 == 0;
    // the one-pass panel kernel holds one chunk (512 or 1024 columns) in registers
    if (vec && !trans && kch == SPLIT_KCH)
        split3_panel_kernel<1><<<dim3((unsigned)ceil_div(R, SPP_ROWS), g.y), 256, 0, s>>>(a);
    else if (vec && !trans)
        split3_panel_kernel<2><<<dim3((unsigned)ceil_div(R, SPP_ROWS), g.y), 512, 0, s>>>(a);
    else if (vec && trans)
        split3_vec_kernel<<<g, 256, 0, s>>>(a);
    else
        split_rows_kernel<<<g, 256, 0, s>>>(a);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_PACK, 0.0, (double)R * K * (8.0 + 2.0 * S));
    return GP_OK;
}

}  // namespace gp
