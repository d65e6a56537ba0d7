// trsv_persist.cu -- single-launch blocked triangular solves with the
// Cholesky factor: v = L^{-1} b (Sec. 1, the forward solve of y - mu) and
// alpha = L^{-T} v (the paper's backsolve), for the solves inside the
// log-likelihood and its refinement.
//
// One CTA per 64-row block.  A CTA takes its block from an atomic ticket, so
// every block it depends on was taken by a CTA that is already running or
// done (no deadlock whatever the scheduling order).  It accumulates the
// block's GEMV contribution from each finished block as soon as that block's
// flag is set (bounded wait), then solves its 64 x 64 diagonal triangle in
// one warp (solution in registers, broadcast by shuffles) and publishes the
// result: store, __threadfence, flag.  L is read once per solve; the chain
// of diagonal solves is the only serial part.  A wait that gives up (1 s)
// sets *info = -1 and the CTA returns without publishing.
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

__device__ __forceinline__ void publish(double *b, int64_t r0, int bs, double v0, double v1,
                                        int *flag) {
    const int l = threadIdx.x & 31;
    if (l < bs) b[r0 + l] = v0;
    if (l + 32 < bs) b[r0 + l + 32] = v1;
    __threadfence();
    __syncwarp();
    if (l == 0) atomicExch(flag, 1);
}

// forward: rows of block i need v_j for every j < i
__global__ void __launch_bounds__(256) trsv_fwd_persist_kernel(const double *__restrict__ L,
                                                               int64_t ld, int64_t n, double *b,
                                                               int *sync, int64_t *info,
                                                               const int *skip) {
    __shared__ int s_blk, s_ok;
    __shared__ double xs[PB];
    __shared__ double part[4][PB];
    __shared__ double Ld[PB * (PB + 1)];  // diagonal tile, Ld[c (PB+1) + r] = L[r0+r, r0+c]
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
    // the diagonal tile and its pivots' reciprocals do not depend on other
    // blocks: stage them while the earlier blocks are still being solved
    for (int e = tid; e < PB * PB; e += blockDim.x) {
        const int rr = e & (PB - 1), cc = e >> 6;
        Ld[cc * (PB + 1) + rr] = (rr < bs && cc < bs && rr >= cc) ? L[(r0 + rr) + (r0 + cc) * ld] : 0.0;
    }
    __syncthreads();
    if (tid < bs) rinv[tid] = 1.0 / Ld[tid * (PB + 1) + tid];
    double acc = 0.0;
    for (int j = 0; j < i; ++j) {
        if (tid == 0) s_ok = wait_flag(&sync[1 + j], info);
        __syncthreads();
        if (!s_ok) return;
        if (tid < PB) xs[tid] = reinterpret_cast<volatile double *>(b)[(int64_t)j * PB + tid];
        __syncthreads();
        if (r < bs) {
            const double *p = L + (r0 + r) + ((int64_t)j * PB + cg * 16) * ld;
#pragma unroll 8
            for (int c = 0; c < 16; ++c) acc = fma(p[c * ld], xs[cg * 16 + c], acc);
        }
        __syncthreads();
    }
    part[cg][r] = acc;
    __syncthreads();
    if (tid >= 32) return;
    const int l = tid;
    double v0 = 0.0, v1 = 0.0;
    if (l < bs) v0 = b[r0 + l] - (part[0][l] + part[1][l] + part[2][l] + part[3][l]);
    if (l + 32 < bs)
        v1 = b[r0 + l + 32] - (part[0][l + 32] + part[1][l + 32] + part[2][l + 32] + part[3][l + 32]);
    for (int c = 0; c < bs; ++c) {
        const double mine = (c < 32) ? v0 : v1;
        const double xc = __shfl_sync(0xffffffffu, mine, c & 31) * rinv[c];
        if (l == (c & 31)) {
            if (c < 32) v0 = xc; else v1 = xc;
        }
        const double *col = Ld + c * (PB + 1);
        if (l > c) v0 -= col[l] * xc;
        if (l + 32 > c) v1 -= col[l + 32] * xc;
    }
    publish(b, r0, bs, v0, v1, &sync[1 + i]);
}

// backward: block i needs alpha_j for every j > i; tickets run from the last
// block to the first
__global__ void __launch_bounds__(256) trsv_bwd_persist_kernel(const double *__restrict__ L,
                                                               int64_t ld, int64_t n, double *b,
                                                               int *sync, int64_t *info,
                                                               const int *skip) {
    __shared__ int s_blk, s_ok;
    __shared__ double xs[PB];
    __shared__ double part[PB];
    __shared__ double Ld[PB * (PB + 1)];  // diagonal tile, Ld[c (PB+1) + r] = L[r0+r, r0+c]
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
    for (int e = tid; e < PB * PB; e += blockDim.x) {
        const int rr = e & (PB - 1), cc = e >> 6;
        Ld[cc * (PB + 1) + rr] = (rr < bs && cc < bs && rr >= cc) ? L[(r0 + rr) + (r0 + cc) * ld] : 0.0;
    }
    __syncthreads();
    if (tid < bs) rinv[tid] = 1.0 / Ld[tid * (PB + 1) + tid];
    // lane partials for the 8 columns (of this block) owned by this warp
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
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
        for (int q = 0; q < 8; ++q) {
            const int c = warp + 8 * q;  // column of block i
            if (c < bs) {
                const double *col = L + j0 + (r0 + c) * ld;
                double a = 0.0;
                if (lane < bj) a = col[lane] * x0;
                if (lane + 32 < bj) a = fma(col[lane + 32], x1, a);
                acc[q] += a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double a = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) part[warp + 8 * q] = a;
    }
    __syncthreads();
    if (tid >= 32) return;
    const int l = tid;
    double v0 = 0.0, v1 = 0.0;
    if (l < bs) v0 = b[r0 + l] - part[l];
    if (l + 32 < bs) v1 = b[r0 + l + 32] - part[l + 32];
    for (int c = bs - 1; c >= 0; --c) {
        const double mine = (c < 32) ? v0 : v1;
        const double xc = __shfl_sync(0xffffffffu, mine, c & 31) * rinv[c];
        if (l == (c & 31)) {
            if (c < 32) v0 = xc; else v1 = xc;
        }
        // row c of the tile: L[r0+c, r0+l] = Ld[l (PB+1) + c]
        if (l < c) v0 -= Ld[l * (PB + 1) + c] * xc;
        if (l + 32 < c) v1 -= Ld[(l + 32) * (PB + 1) + c] * xc;
    }
    publish(b, r0, bs, v0, v1, &sync[1 + i]);
}

size_t trsv_sync_ints(int64_t n) { return (size_t)ceil_div(n, PB) + 2; }

int trsv_persist(const double *L, int64_t ld, int64_t n, int trans, double *b, int *sync,
                 int64_t *info, const int *skip, cudaStream_t s) {
    const int64_t T = ceil_div(n, PB);
    if (cudaMemsetAsync(sync, 0, sizeof(int) * (T + 1), s) != cudaSuccess) return GP_ERR_CUDA;
    const int ev = prof_start(s);
    if (trans == 0)
        trsv_fwd_persist_kernel<<<(unsigned)T, 256, 0, s>>>(L, ld, n, b, sync, info, skip);
    else
        trsv_bwd_persist_kernel<<<(unsigned)T, 256, 0, s>>>(L, ld, n, b, sync, info, skip);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_SOLVE, 0.0, 8.0 * (double)n * (double)(n + 1) / 2.0);
    return GP_OK;
}

}  // namespace gp
