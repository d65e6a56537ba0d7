// tc_gemm.cu -- the dense contraction of the trailing update (Sec. 2.1: "most
// of the total work is in the matrix multiplications") on the sm_103a
// tensor cores, with FP64 operands carried as BF16 slices.
//
// Operand splitting.  Each FP64 operand element x is written as a sum of
// S BF16 slices, s_0 = bf16(x), s_1 = bf16(x - s_0), s_2 = bf16(x - s_0 - s_1);
// each slice keeps 8 more significant bits, so three slices carry x to about
// 2^-24 relative.  A product x*y is then the sum of the slice products
// s_p t_q with p + q < S (6 products for S = 3; the dropped ones are below
// 2^-24 relative).  All of them accumulate in one FP32 accumulator in
// tensor memory, so the contraction is FP32-accurate; the factor's FP64
// parts (diagonal blocks, pivots, log-determinant, residuals) stay FP64.
//
// Slice layout.  An operand of R rows and K columns is packed as
// bf16[S][R][K] (K contiguous, "K-major"), read by TMA with a 3-D tensor map
// {K, R, S} in 64 x rows boxes with the 128-byte swizzle, which is the
// canonical K-major SWIZZLE_128B layout the tcgen05 shared-memory
// descriptors address.
//
// Kernel.  One CTA per 128 x 256 output tile, 6 warps:
//   warp 0  TMA producer (one elected thread), 4-stage ring of 48 KB stages;
//   warp 1  TMEM allocation (256 FP32 columns) and the MMA issuer (one
//           thread issues tcgen05.mma.cta_group::1.kind::f16 with BF16
//           inputs, 4 x K16 per stage, and tcgen05.commit to free the stage);
//   warps 2-5  epilogue: tcgen05.ld 32 lanes x 32 columns, then
//           C = beta C + alpha acc in FP64, one row per thread, so each warp
//           store covers 32 consecutive rows of a column (coalesced).
// Every mbarrier wait is bounded; a wait that gives up sets *info = -1 and
// the CTA winds down (waiting, again bounded, for its copies in flight)
// and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "internal.h"
#include "tc_gemm.h"

namespace gp {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_BK = 64;
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 /*barriers*/ + 1024 /*align*/;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr uint32_t WAIT_LIMIT = 1u << 24;  // x ~100 ns backoff: well above any real wait

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 16) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); LBO unused for swizzled K-major; version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(1) << 16;
    d |= static_cast<uint64_t>(1024 >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   TcGemmArgs args) {
    extern __shared__ uint8_t smem_raw[];
    const int tile_m = blockIdx.x, tile_n = blockIdx.y;
    const int64_t row0 = (int64_t)tile_m * TC_BM, col0 = (int64_t)tile_n * TC_BN;
    if (args.lower && col0 >= row0 + TC_BM) return;  // tile strictly above the diagonal
    if (args.info && failed(args.info)) return;

    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    uint8_t *stage_base = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *done = empty + TC_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
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
    const int kt = args.npairs * args.kblocks;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int issued = 0;
        for (int it = 0; it < kt; ++it) {
            const int s = it % TC_STAGES, use = it / TC_STAGES;
            if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
                abort_flag = 1;
                break;
            }
            const int pair = it / args.kblocks, kb = it % args.kblocks;
            uint8_t *a_s = stage_base + s * TC_STAGE_BYTES;
            uint8_t *b_s = a_s + TC_A_BYTES;
            mbar_arrive_expect_tx(&full[s], TC_STAGE_BYTES);
            tma_load_3d(a_s, &tmA, &full[s], kb * TC_BK, (int)row0 + args.a_row_off, args.pa[pair]);
            tma_load_3d(b_s, &tmB, &full[s], kb * TC_BK, (int)col0 + args.b_row_off, args.pb[pair]);
            issued = it + 1;
        }
        // drain: every issued stage must land before the CTA may exit
        for (int it = (issued > TC_STAGES ? issued - TC_STAGES : 0); it < issued; ++it) {
            const int s = it % TC_STAGES, use = it / TC_STAGES;
            mbar_wait(&full[s], use & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = idesc_bf16_f32(TC_BM, TC_BN);
        bool ok = true;
        for (int it = 0; it < kt; ++it) {
            const int s = it % TC_STAGES, use = it / TC_STAGES;
            if (!mbar_wait(&full[s], use & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(stage_base + s * TC_STAGE_BYTES);
            const uint32_t b_addr = a_addr + TC_A_BYTES;
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k) {
                mma_bf16_ss(tmem, sdesc_sw128(a_addr + k * 32), sdesc_sw128(b_addr + k * 32), idesc,
                            (it > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
        }
        if (!ok) abort_flag = 1;
        mma_commit(done);  // arrives once all issued MMAs have completed
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        bool ok = mbar_wait(done, 0);
        tc_fence_after();
        const bool go = __all_sync(0xffffffffu, ok && !abort_flag);
        if (go) {
            const int64_t row = row0 + q * 32 + lane;
            const double alpha = args.alpha, beta = args.beta;
            for (int c0 = 0; c0 < TC_BN; c0 += 32) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(q * 32) << 16) + c0, v);
                if (row >= args.M) continue;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t col = col0 + c0 + j;
                    if (col >= args.N) break;
                    if (args.lower && row < col) continue;
                    double *p = args.C + row + col * args.ldc;
                    double acc = static_cast<double>(__uint_as_float(v[j]));
                    double r = alpha * acc;
                    if (beta != 0.0) r = fma(beta, *p, r);
                    *p = r;
                }
            }
        }
        if (!ok && lane == 0) abort_flag = 1;
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
// Split FP64 -> BF16 slices.
// src(r, k) = src[r + k ld]          (trans = 0: rows of the operand are rows
//                                     of the column-major source)
// src(r, k) = src[k + r ld]          (trans = 1: rows are source columns)
// lower_mask: zero entries with source row < source column (a triangular
// source whose upper part holds stale data).
// dst[p][r][k], p < S, shape S x R x K (K contiguous); columns k >= Kvalid
// are written as zeros (K padded to the 64-column MMA step).  32 x 32 tiles are
// transposed through shared memory so both sides stay coalesced.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) split_bf16_kernel(const double *__restrict__ src, int64_t ld,
                                                          int64_t R, int64_t K, int64_t Kvalid,
                                                          int trans, int64_t diag_off,
                                                          int lower_mask, int S,
                                                          __nv_bfloat16 *__restrict__ dst) {
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty 0..7
    // load a 32 x 32 block indexed [r][k]
    for (int i = ty; i < 32; i += 8) {
        double v = 0.0;
        if (trans == 0) {
            const int64_t r = r0 + tx, k = k0 + i;  // source rows contiguous: r fastest
            if (r < R && k < Kvalid) {
                v = src[r + k * ld];
                if (lower_mask && r + diag_off < k) v = 0.0;
            }
            t[tx][i] = v;
        } else {
            const int64_t r = r0 + i, k = k0 + tx;  // source column r, row k: k fastest
            if (r < R && k < Kvalid) {
                v = src[k + r * ld];
                if (lower_mask && k + diag_off < r) v = 0.0;
            }
            t[i][tx] = v;
        }
    }
    __syncthreads();
    const int64_t RK = R * K;
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i, k = k0 + tx;
        if (r >= R || k >= K) continue;
        double x = t[i][tx];
        __nv_bfloat16 *d = dst + r * K + k;
        for (int p = 0; p < S; ++p) {
            __nv_bfloat16 h = __double2bfloat16(x);
            d[p * RK] = h;
            x -= static_cast<double>(__bfloat162float(h));
        }
    }
}

int split_bf16(const double *src, int64_t ld, int64_t R, int64_t K, int64_t Kvalid, int trans,
               int64_t diag_off, int lower_mask, int S, __nv_bfloat16 *dst, cudaStream_t s) {
    if (R <= 0 || K <= 0) return GP_OK;
    dim3 g((unsigned)ceil_div(K, 32), (unsigned)ceil_div(R, 32));
    split_bf16_kernel<<<g, 256, 0, s>>>(src, ld, R, K, Kvalid, trans, diag_off, lower_mask, S, dst);
    GP_LAUNCH_CHECK();
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

static int make_slice_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t R, int64_t K, int S,
                          int box_rows) {
    auto fn = encode_fn();
    if (!fn) return GP_ERR_CUDA;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (K * 2) % 16) return GP_ERR_INVALID;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)(R * K * 2)};
    cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GP_OK : GP_ERR_CUDA;
}

int tc_gemm(const TcOperand &A, const TcOperand &B, int64_t M, int64_t N, int64_t K, double alpha,
            double beta, double *C, int64_t ldc, int lower, int nslices, int64_t *info,
            cudaStream_t s) {
    if (M <= 0 || N <= 0) return GP_OK;
    if (K % TC_BK) return GP_ERR_INVALID;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_SMEM) != cudaSuccess)
            return GP_ERR_CUDA;
        attr_set = true;
    }
    CUtensorMap ma, mb;
    GP_TRY(make_slice_map(&ma, A.slices, A.rows, A.K, A.S, TC_BM));
    GP_TRY(make_slice_map(&mb, B.slices, B.rows, B.K, B.S, TC_BN));
    TcGemmArgs a{};
    a.C = C;
    a.ldc = ldc;
    a.M = M;
    a.N = N;
    a.alpha = alpha;
    a.beta = beta;
    a.kblocks = (int)(K / TC_BK);
    a.lower = lower;
    a.info = info;
    a.a_row_off = (int)A.row_off;
    a.b_row_off = (int)B.row_off;
    int np = 0;
    for (int p = 0; p < nslices; ++p)
        for (int q = 0; p + q < nslices; ++q) {
            a.pa[np] = p;
            a.pb[np] = q;
            ++np;
        }
    a.npairs = np;
    dim3 g((unsigned)ceil_div(M, TC_BM), (unsigned)ceil_div(N, TC_BN));
    tc_gemm_kernel<<<g, 192, TC_SMEM, s>>>(ma, mb, a);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

}  // namespace gp
