// tc_gemm.cu -- the dense contractions of the blocked Cholesky (Sec. 2.1:
// "most of the total work is in the matrix multiplications") and of the
// gradient's inverse, on the sm_103a tensor cores, with FP64 operands
// carried as BF16 slices.
//
// Operand splitting (row-scaled).  For operand row r let 2^e_r bound its
// entries over the packed K range.  Each FP64 entry x becomes three BF16
// slices:
//   s0 = round(x 2^{7-e_r}) 2^{e_r-7}     an integer in [-128, 128] times a
//                                         per-row power of two (exact in BF16)
//   s1 = bf16(x - s0),  s2 = bf16(x - s0 - s1)
// so x = s0 + s1 + s2 to about 2^-26 of the row's largest entry.  A product
// sum over k is the sum of slice products s_p t_q with p + q < 3 (the
// dropped ones are below 2^-25 of the row maxima).  The leading products
// s0 t0 are integers times one common power of two for a given output
// (r, c); their sums stay below 2^24 units for K <= 1024, so the FP32
// tensor-core accumulator holds them exactly however it rounds.  They go to
// their own accumulator ("hi"); the five smaller products share a second one
// ("lo"), whose rounding is 2^-7 smaller.  The epilogue adds hi + lo.
//
// Kernel.  Persistent: one CTA per SM walks a static tile schedule of
// 128 x 128 output tiles (grouped 16 tile-rows at a time so the operand
// tiles in flight stay in L2).  6 warps:
//   warp 0     TMA producer (one thread): a 6-stage ring of 32 KB stages
//              (A and B 128 x 64 BF16 boxes, 128-byte swizzle).
//   warp 1     TMEM owner (512 columns = 2 tile buffers x {hi, lo}) and MMA
//              issuer (one thread): tcgen05.mma.cta_group::1.kind::f16,
//              128 x 128 x 16 per instruction; tcgen05.commit frees stages
//              and hands finished accumulators to the epilogue.
//   warps 2-5  epilogue: tcgen05.ld of hi and lo (32 lanes x 32 columns),
//              output in FP64 (C = beta C + alpha acc) or FP32 (C += alpha
//              acc), one row per thread so that every warp access covers 32
//              consecutive rows of one column; all loads of a 32-column chunk
//              are issued before any store.  The two TMEM buffers let the
//              epilogue of one tile overlap the MMAs of the next.
// Every mbarrier wait is bounded (1 s); a wait that gives up sets
// *info = -1, the roles wind down (the producer waits, bounded, for its
// copies in flight) and TMEM is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "internal.h"
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
constexpr int TC_MAX_PAIRS = 6;

struct TcGemmArgs {
    void *C;
    int64_t ldc;
    int fp32;
    double alpha, beta;
    int lower;
    int64_t diag_off;
    int64_t M, N;
    int a_row_off, b_row_off, a_k_off, b_k_off;
    int kblocks;
    int tri_k;
    int64_t tri_off;
    int tiles_m, tiles_n;
    int npairs;
    int pa[TC_MAX_PAIRS], pb[TC_MAX_PAIRS];
    int64_t *info;
};

struct TileInfo {
    int tm, tn, kb_lo, kb_hi;
    bool skip;
};

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

__global__ void __launch_bounds__(192, 1)
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
            mbar_init(&tempty[b], 4);
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
            for (int p = 0; p < args.npairs && ok; ++p) {
                for (int kb = ti.kb_lo; kb < ti.kb_hi; ++kb, ++it) {
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
        if (!ok) abort_flag = 1;
        // drain: copies still in flight must land before the CTA exits
        for (uint32_t j = (it > TC_STAGES ? it - TC_STAGES : 0); j < it; ++j)
            mbar_wait(&full[j % TC_STAGES], (j / TC_STAGES) & 1);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = idesc_bf16_f32(TC_BM, TC_BN);
        uint32_t it = 0, local = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const uint32_t buf = local & 1, u = local >> 1;
            if (u > 0 && !mbar_wait(&tempty[buf], (u - 1) & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            for (int p = 0; p < args.npairs && ok; ++p) {
                const uint32_t acc = tmem + (buf * 2 + (p > 0 ? 1 : 0)) * TC_BN;
                const bool first_of_acc = (p <= 1);
                for (int kb = ti.kb_lo; kb < ti.kb_hi; ++kb, ++it) {
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
                        const uint32_t accumulate = (first_of_acc && kb == ti.kb_lo && k == 0) ? 0u : 1u;
                        mma_bf16_ss(acc, sdesc_sw128(a_addr + k * 32), sdesc_sw128(b_addr + k * 32),
                                    idesc, accumulate);
                    }
                    mma_commit(&empty[s]);
                }
            }
            mma_commit(&tfull[buf]);
            ++local;
        }
        if (!ok) abort_flag = 1;
        mma_commit(drain);
        mbar_wait(drain, 0);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        uint32_t local = 0;
        const float alpha_f = static_cast<float>(args.alpha);
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const TileInfo ti = tile_at(args, t);
            if (ti.skip) continue;
            const uint32_t buf = local & 1, u = local >> 1;
            bool ok = mbar_wait(&tfull[buf], u & 1);
            ok = __all_sync(0xffffffffu, ok) && !abort_flag;
            if (!ok) {
                if (lane == 0) abort_flag = 1;
                break;
            }
            tc_fence_after();
            const bool has_acc = ti.kb_lo < ti.kb_hi;
            const bool has_lo = args.npairs > 1;
            const int64_t row = (int64_t)ti.tm * TC_BM + q * 32 + lane;
            const bool row_ok = row < args.M;
            for (int c0 = 0; c0 < TC_BN; c0 += 32) {
                uint32_t hi[32], lo[32];
                if (has_acc) {
                    const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + c0;
                    tmem_ld_32x32b_x32(base + (buf * 2) * TC_BN, hi);
                    if (has_lo) tmem_ld_32x32b_x32(base + (buf * 2 + 1) * TC_BN, lo);
                    tmem_ld_wait();
                }
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float h = has_acc ? __uint_as_float(hi[j]) : 0.0f;
                    float l = (has_acc && has_lo) ? __uint_as_float(lo[j]) : 0.0f;
                    v[j] = h + l;
                }
                const int64_t colb = (int64_t)ti.tn * TC_BN + c0;
                bool okc[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t col = colb + j;
                    okc[j] = row_ok && col < args.N && (!args.lower || row + args.diag_off >= col);
                }
                if (args.fp32) {
                    float *base = static_cast<float *>(args.C) + row + colb * args.ldc;
                    float old[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) old[j] = okc[j] ? base[j * args.ldc] : 0.0f;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (okc[j]) base[j * args.ldc] = fmaf(alpha_f, v[j], old[j]);
                } else {
                    double *base = static_cast<double *>(args.C) + row + colb * args.ldc;
                    if (args.beta != 0.0) {
                        double old[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) old[j] = okc[j] ? base[j * args.ldc] : 0.0;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (okc[j])
                                base[j * args.ldc] =
                                    fma(args.beta, old[j], args.alpha * static_cast<double>(v[j]));
                    } else if (args.alpha == 1.0 || args.alpha == -1.0) {
                        const float sg = args.alpha > 0.0 ? 1.0f : -1.0f;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (okc[j]) base[j * args.ldc] = static_cast<double>(sg * v[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (okc[j]) base[j * args.ldc] = args.alpha * static_cast<double>(v[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            ++local;
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
    int S;
    __nv_bfloat16 *dst;
    int64_t dst_rows, dst_kld, dst_row_off, dst_k_off;
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

// x = hi + lo with integer operations only (the FP64 pipe is the scarce one
// on this part): hi keeps the top 24 significant bits (truncated), lo the
// remaining 29 rounded to FP32.  Magnitudes below 2^-126 map to 0 and lo
// parts below 2^-126 are dropped (negligible next to the row bounds used).
__device__ __forceinline__ void f64_hi_lo(unsigned long long u, float &hi, float &lo) {
    const unsigned int sign = static_cast<unsigned int>(u >> 32) & 0x80000000u;
    const int E = static_cast<int>((u >> 52) & 0x7FF);
    const int ef = E - 1023 + 127;
    hi = 0.0f;
    lo = 0.0f;
    if (E == 0 || ef <= 0) return;
    if (ef >= 255) {
        hi = __int_as_float(sign | 0x7F800000u);
        return;
    }
    const unsigned long long mant = u & 0x000FFFFFFFFFFFFFull;
    hi = __int_as_float(sign | (static_cast<unsigned int>(ef) << 23) |
                        static_cast<unsigned int>(mant >> 29));
    const int es = E - 1075;  // weight of the mantissa's last bit
    if (es >= -126) {
        const float lf = __uint2float_rn(static_cast<unsigned int>(mant & 0x1FFFFFFFull));
        lo = __int_as_float(__float_as_int(lf * __int_as_float((es + 127) << 23)) | sign);
    }
}

// s0, s1, s2 for one entry, given the row's scale 2^{7-e} (sc) and 2^{e-7} (isc).
__device__ __forceinline__ void split3(unsigned long long u, float sc, float isc,
                                       __nv_bfloat16 (&s)[3]) {
    float xh, xl;
    f64_hi_lo(u, xh, xl);
    const float q = rintf(xh * sc);
    const float s0 = q * isc;
    const float r1 = (xh - s0) + xl;
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    s[0] = __float2bfloat16_rn(s0);
    s[1] = b1;
    s[2] = __float2bfloat16_rn(r2);
}

constexpr int64_t SPLIT_KCH = 512;  // K chunk of one CTA (and of one row bound)

__global__ void __launch_bounds__(256) split_rows_kernel(SplitArgs a) {
    __shared__ unsigned long long pmax[8][32];
    __shared__ float sc_s[32], isc_s[32];
    __shared__ unsigned short tile[3][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    // this CTA's K chunk; each (row, chunk) gets its own bound 2^e
    const int64_t kb = (int64_t)blockIdx.y * SPLIT_KCH;
    const int64_t ke = min(a.K, kb + SPLIT_KCH);
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
    }
    __syncthreads();
    const int64_t slice = a.dst_rows * a.dst_kld;
    __nv_bfloat16 *d0 = a.dst + (a.dst_row_off + r0) * a.dst_kld + a.dst_k_off;
    if (a.trans == 0) {
        for (int64_t kc = kb; kc < ke; kc += 32) {
            // lane = row: coalesced FP64 reads down each column
            for (int i = warp; i < 32; i += 8) {
                __nv_bfloat16 s[3];
                split3(split_get(a, r0 + lane, kc + i), sc_s[lane], isc_s[lane], s);
#pragma unroll
                for (int p = 0; p < 3; ++p) tile[p][i][lane] = __bfloat16_as_ushort(s[p]);
            }
            __syncthreads();
            // lane = k: coalesced BF16 writes along each row
            for (int i = warp; i < 32; i += 8) {
                const int64_t r = r0 + i, k = kc + lane;
                if (r < a.R && k < ke) {
                    for (int p = 0; p < a.S; ++p)
                        d0[p * slice + (int64_t)i * a.dst_kld + k] =
                            __ushort_as_bfloat16(tile[p][lane][i]);
                }
            }
            __syncthreads();
        }
    } else {
        for (int i = warp; i < 32; i += 8) {
            const int64_t r = r0 + i;
            if (r >= a.R) continue;
            for (int64_t k = kb + lane; k < ke; k += 32) {
                __nv_bfloat16 s[3];
                split3(split_get(a, r, k), sc_s[i], isc_s[i], s);
                for (int p = 0; p < a.S; ++p) d0[p * slice + (int64_t)i * a.dst_kld + k] = s[p];
            }
        }
    }
}

int split_rows(const double *src, int64_t ld, int64_t R, int64_t K, int64_t Kvalid, int trans,
               int64_t diag_off, int lower_mask, int S, __nv_bfloat16 *dst, int64_t dst_rows,
               int64_t dst_kld, int64_t dst_row_off, int64_t dst_k_off, cudaStream_t s) {
    if (R <= 0 || K <= 0) return GP_OK;
    if (S < 1 || S > 3 || dst_row_off + R > dst_rows || dst_k_off + K > dst_kld)
        return GP_ERR_INVALID;
    SplitArgs a{src, ld, R, K, Kvalid < K ? Kvalid : K, trans, diag_off, lower_mask, S, dst,
                dst_rows, dst_kld, dst_row_off, dst_k_off};
    const int ev = prof_start(s);
    dim3 g((unsigned)ceil_div(R, 32), (unsigned)ceil_div(K, SPLIT_KCH));
    split_rows_kernel<<<g, 256, 0, s>>>(a);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_PACK, 0.0, (double)R * K * (8.0 + 2.0 * S));
    return GP_OK;
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

static int make_slice_map(CUtensorMap *map, const TcOperand &op, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return GP_ERR_CUDA;
    if ((reinterpret_cast<uintptr_t>(op.slices) & 15) || (op.Kld % TC_BK)) return GP_ERR_INVALID;
    cuuint64_t dims[3] = {(cuuint64_t)op.Kld, (cuuint64_t)op.rows, (cuuint64_t)op.S};
    cuuint64_t strides[2] = {(cuuint64_t)op.Kld * 2, (cuuint64_t)(op.rows * op.Kld * 2)};
    cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(op.slices),
                    dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
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
    if (A.k_off + K > A.Kld || B.k_off + K > B.Kld || A.S != B.S) return GP_ERR_INVALID;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_SMEM) != cudaSuccess)
            return GP_ERR_CUDA;
        attr_set = true;
    }
    CUtensorMap ma, mb;
    GP_TRY(make_slice_map(&ma, A, TC_BM));
    GP_TRY(make_slice_map(&mb, B, TC_BN));
    TcGemmArgs a{};
    a.C = out.C;
    a.ldc = out.ldc;
    a.fp32 = out.fp32;
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
    a.tiles_m = (int)ceil_div(M, TC_BM);
    a.tiles_n = (int)ceil_div(N, TC_BN);
    a.info = info;
    int np = 0;
    for (int d = 0; d < A.S; ++d)      // pairs in order of decreasing size:
        for (int p = 0; p <= d; ++p) { // (0,0) first, it owns the "hi" accumulator
            a.pa[np] = p;
            a.pb[np] = d - p;
            ++np;
        }
    a.npairs = np;
    const int64_t ntiles = (int64_t)a.tiles_m * a.tiles_n;
    const int sms = num_sms();
    const int grid = (int)(ntiles < sms ? ntiles : (sms > 0 ? sms : 148));
    const int ev = prof_start(s);
    tc_gemm_kernel<<<grid, 192, TC_SMEM, s>>>(ma, mb, a);
    GP_LAUNCH_CHECK();
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
        prof_stop(ev, s, GP_PROF_CONTRACT, 2.0 * np * useful, 0.0);
    }
    return GP_OK;
}

}  // namespace gp
