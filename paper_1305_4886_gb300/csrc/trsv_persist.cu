// trsv_persist.cu -- single-launch blocked triangular solves with the
// Cholesky factor: v = L^{-1} b (Sec. 1, the forward solve of y - mu) and
// alpha = L^{-T} v (the paper's backsolve), for the solves inside the
// log-likelihood and its refinement.
//
// One CTA per 64-row block.  A CTA takes its block from an atomic ticket, so
// every block it depends on was taken by a CTA that is already running or
// done (no deadlock whatever the scheduling order).  It accumulates the
// block's GEMV contribution from each finished block as soon as that block's
// flag is set (bounded wait; the tile's values are loaded before the wait),
// then applies the inverse of its 64 x 64 diagonal triangle, formed while it
// waited, and publishes the result: store, __threadfence, flag.  L is read
// once per solve; the chain of diagonal products is the only serial part.
// A wait that gives up (1 s) sets *info = -1 and the CTA returns without
// publishing.
#include <mutex>

#include "internal.h"
#include "tc_ptx.cuh"

namespace gp {

constexpr int PB = 64;

// Bounded wait on a publication flag (read with volatile loads).
__device__ __forceinline__ bool wait_flag(const int *flag, int64_t *info) {
    if (*reinterpret_cast<const volatile int *>(flag)) {
        __threadfence();
        return true;
    }
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 0;; ++i) {
        if (*reinterpret_cast<const volatile int *>(flag)) {
            __threadfence();
            return true;
        }
        __nanosleep(64);
        if ((i & 63) == 0 && globaltimer_ns() - t0 > WAIT_NS) {
            if (info) set_info(info, -1);
            return false;
        }
    }
}

// Inverse of the block's 64 x 64 lower diagonal tile, formed while the block
// waits for its turn (no dependence on other blocks).  Ld[c (PB+1) + r] =
// L_rc on entry (rows / columns >= bs: the identity); on exit Wd holds
// W = L^{-1} in the same layout and Ld is overwritten.  Elimination on
// Y = I: with M_lc = L_lc / L_ll, for l descending, Y_c -= Y_l M_lc (c < l);
// then W_c = Y_c / L_cc.
__device__ void diag_inverse(double *Ld, double *Wd, double *rinv) {
    const int tid = threadIdx.x;
    if (tid < PB) rinv[tid] = 1.0 / Ld[tid * (PB + 1) + tid];
    __syncthreads();
    for (int e = tid; e < PB * PB; e += blockDim.x) {
        const int r = e & (PB - 1), c = e >> 6;
        if (r > c) Ld[c * (PB + 1) + r] *= rinv[r];
        Wd[c * (PB + 1) + r] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int l = PB - 1; l > 0; --l) {
        // column l of Y is zero above row l: rows l.. only (exact zeros skipped)
        const int nr = PB - l;
        for (int e = tid; e < l * nr; e += blockDim.x) {
            const int c = e / nr, r = l + (e - c * nr);
            Wd[c * (PB + 1) + r] = fma(-Wd[l * (PB + 1) + r], Ld[c * (PB + 1) + l], Wd[c * (PB + 1) + r]);
        }
        __syncthreads();
    }
    for (int e = tid; e < PB * PB; e += blockDim.x) {
        const int r = e & (PB - 1), c = e >> 6;
        Wd[c * (PB + 1) + r] = (r >= c) ? Wd[c * (PB + 1) + r] * rinv[c] : 0.0;
    }
    __syncthreads();
}

// Store the block's solution (threads < bs), then raise its flag.
__device__ __forceinline__ void publish_block(double *b, int64_t r0, int bs, double v, int *flag) {
    if (threadIdx.x < bs) b[r0 + threadIdx.x] = v;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(flag, 1);
}

__device__ __forceinline__ void load_diag_tile(const double *L, int64_t ld, int64_t r0, int bs,
                                               double *Ld) {
    for (int e = threadIdx.x; e < PB * PB; e += blockDim.x) {
        const int rr = e & (PB - 1), cc = e >> 6;
        double v = 0.0;
        if (rr < bs && cc < bs) v = (rr >= cc) ? L[(r0 + rr) + (r0 + cc) * ld] : 0.0;
        else if (rr == cc) v = 1.0;
        Ld[cc * (PB + 1) + rr] = v;
    }
    __syncthreads();
}

// forward: rows of block i need v_j for every j < i
__global__ void __launch_bounds__(256) trsv_fwd_persist_kernel(const double *__restrict__ L,
                                                               int64_t ld, int64_t n, double *b,
                                                               int *sync, int64_t *info,
                                                               const int *skip) {
    __shared__ int s_blk, s_ok;
    __shared__ double xs[PB];
    __shared__ double part[4][PB];
    extern __shared__ double trsv_dyn[];  // Ld, Wd: PB (PB + 1) each
    double *Ld = trsv_dyn, *Wd = trsv_dyn + PB * (PB + 1);
    __shared__ double rinv[PB];
    if ((skip && *skip) || failed(info)) return;
    const int tid = threadIdx.x;
    const int T = (int)ceil_div(n, PB);
    if (tid == 0) s_blk = atomicAdd(&sync[0], 1);
    __syncthreads();
    const int i = s_blk;
    if (i >= T) return;
    const int64_t r0 = (int64_t)i * PB;
    const int bs = (int)min((int64_t)PB, n - r0);
    const int r = tid & (PB - 1), cg = tid >> 6;
    load_diag_tile(L, ld, r0, bs, Ld);
    diag_inverse(Ld, Wd, rinv);
    // off-diagonal tiles: each tile's 16 values per thread are loaded before
    // the wait for the block that owns its solution
    double acc = 0.0;
    double lv[16];
    auto load_tile = [&](int j) {
        const double *p = L + (r0 + r) + ((int64_t)j * PB + cg * 16) * ld;
#pragma unroll
        for (int c = 0; c < 16; ++c) lv[c] = (r < bs) ? p[c * ld] : 0.0;
    };
    if (i > 0) load_tile(0);
    for (int j = 0; j < i; ++j) {
        if (tid == 0) s_ok = wait_flag(&sync[1 + j], info);
        __syncthreads();
        if (!s_ok) return;
        if (tid < PB) xs[tid] = reinterpret_cast<volatile double *>(b)[(int64_t)j * PB + tid];
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 16; ++c) acc = fma(lv[c], xs[cg * 16 + c], acc);
        if (j + 1 < i) load_tile(j + 1);
        __syncthreads();
    }
    part[cg][r] = acc;
    __syncthreads();
    if (tid < PB) xs[tid] = (tid < bs) ? b[r0 + tid] - (part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid]) : 0.0;
    __syncthreads();
    // v_i = W (b_i - sum): row r over columns 16 cg .. (c <= r)
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const int cc = cg * 16 + c;
        if (cc <= r) v = fma(Wd[cc * (PB + 1) + r], xs[cc], v);
    }
    part[cg][r] = v;
    __syncthreads();
    const double x = (tid < PB) ? part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid] : 0.0;
    publish_block(b, r0, bs, x, &sync[1 + i]);
}

// backward: rows of block i need alpha_j for every j > i (column blocks of L)
__global__ void __launch_bounds__(256) trsv_bwd_persist_kernel(const double *__restrict__ L,
                                                               int64_t ld, int64_t n, double *b,
                                                               int *sync, int64_t *info,
                                                               const int *skip) {
    __shared__ int s_blk, s_ok;
    __shared__ double xs[PB];
    __shared__ double part[4][PB];
    extern __shared__ double trsv_dyn[];  // Ld, Wd: PB (PB + 1) each
    double *Ld = trsv_dyn, *Wd = trsv_dyn + PB * (PB + 1);
    __shared__ double rinv[PB];
    if ((skip && *skip) || failed(info)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = (int)ceil_div(n, PB);
    if (tid == 0) s_blk = atomicAdd(&sync[0], 1);
    __syncthreads();
    const int t = s_blk;
    if (t >= T) return;
    const int i = T - 1 - t;
    const int64_t r0 = (int64_t)i * PB;
    const int bs = (int)min((int64_t)PB, n - r0);
    load_diag_tile(L, ld, r0, bs, Ld);
    diag_inverse(Ld, Wd, rinv);
    // lane partials for the 8 columns (of this block) owned by this warp
    double acc[8];
    double lv[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    auto load_tile = [&](int j) {
        const int64_t j0 = (int64_t)j * PB;
        const int bj = (int)min((int64_t)PB, n - j0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = warp + 8 * q;  // column of block i
            const double *col = L + j0 + (r0 + c) * ld;
            lv[2 * q] = (c < bs && lane < bj) ? col[lane] : 0.0;
            lv[2 * q + 1] = (c < bs && lane + 32 < bj) ? col[lane + 32] : 0.0;
        }
    };
    if (i < T - 1) load_tile(T - 1);
    for (int j = T - 1; j > i; --j) {
        if (tid == 0) s_ok = wait_flag(&sync[1 + j], info);
        __syncthreads();
        if (!s_ok) return;
        const int64_t j0 = (int64_t)j * PB;
        const int bj = (int)min((int64_t)PB, n - j0);
        if (tid < PB) xs[tid] = tid < bj ? reinterpret_cast<volatile double *>(b)[j0 + tid] : 0.0;
        __syncthreads();
        const double x0 = xs[lane], x1 = xs[lane + 32];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += fma(lv[2 * q + 1], x1, lv[2 * q] * x0);
        if (j - 1 > i) load_tile(j - 1);
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double a = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) part[0][warp + 8 * q] = a;
    }
    __syncthreads();
    if (tid < PB) xs[tid] = (tid < bs) ? b[r0 + tid] - part[0][tid] : 0.0;
    __syncthreads();
    // alpha_i = W^T (b_i - sum): row r over columns c >= r of W^T, i.e. W(c, r)
    const int r = tid & (PB - 1), cg = tid >> 6;
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const int cc = cg * 16 + c;
        if (cc >= r) v = fma(Wd[r * (PB + 1) + cc], xs[cc], v);
    }
    __syncthreads();
    part[cg][r] = v;
    __syncthreads();
    const double x = (tid < PB) ? part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid] : 0.0;
    publish_block(b, r0, bs, x, &sync[1 + i]);
}

size_t trsv_sync_ints(int64_t n) { return (size_t)ceil_div(n, PB) + 2; }

int trsv_persist(const double *L, int64_t ld, int64_t n, int trans, double *b, int *sync,
                 int64_t *info, const int *skip, cudaStream_t s) {
    const int64_t T = ceil_div(n, PB);
    if (cudaMemsetAsync(sync, 0, sizeof(int) * (T + 1), s) != cudaSuccess) return GP_ERR_CUDA;
    const int ev = prof_start(s);
    constexpr int dyn = 2 * PB * (PB + 1) * (int)sizeof(double);
    // the shared-memory attribute, set once per device (host threads may race here)
    static std::mutex attr_mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(attr_mu);
        if (!attr_set[dev]) {
            if (cudaFuncSetAttribute(trsv_fwd_persist_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess ||
                cudaFuncSetAttribute(trsv_bwd_persist_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
                return GP_ERR_CUDA;
            attr_set[dev] = true;
        }
    }
    if (trans == 0)
        trsv_fwd_persist_kernel<<<(unsigned)T, 256, dyn, s>>>(L, ld, n, b, sync, info, skip);
    else
        trsv_bwd_persist_kernel<<<(unsigned)T, 256, dyn, s>>>(L, ld, n, b, sync, info, skip);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_SOLVE, 0.0, 8.0 * (double)n * (double)(n + 1) / 2.0);
    return GP_OK;
}

}  // namespace gp
