// batch_dag.h -- shared pieces of the batched task-graph launches: the
// per-problem descriptor, the local task lists and their decoding, the
// bounded flag waits, and the FP64 64 x 64 tile routines (the FP64 form's
// tasks, and the diagonal-tile factorisation of the tensor-core form).
#pragma once

#include "internal.h"
#include "kern.cuh"
#include "tc_ptx.cuh"

namespace gp {

constexpr int DB = 64;                  // tile order
constexpr int DLD = DB + 1;             // shared-memory leading dimension
constexpr int DAG_THREADS = 256;
constexpr int DAG_ROUNDS = 1024;        // rounds of the proportional merge
constexpr uint64_t DAG_WAIT_NS = 20ull * 1000 * 1000 * 1000;  // 20 s per wait
constexpr uint32_t DAG_WAIT_POLLS = 1u << 30;

enum DagTaskType { DT_CHOL = 0, DT_SOLVE = 1, DT_TRTRI = 2, DT_LG = 3, DT_FINAL = 4 };

// Per-problem descriptor (device copy in the workspace).
struct DagProb {
    const double2 *x;
    const double *y;
    const double *mu;  // nullable
    double *A;         // FP64 form: L tiles, packed lower (tile (i, j) column-major, 64 x 64)
    double *X;         // FP64 form: L^{-1} tiles, same layout
    double *vec;       // FP64: r, v, alpha (3 m); mixed: r, alpha, s, t (4 m)
    double *part;      // logdet shares (T), gradient shares (3 per tile); mixed: + residual
                       // shares (4 T) and refinement statistics (4)
    int *flag;         // see dag_nflags
    double *out;       // 4 values
    double *grad;      // 3 values
    int64_t *info;
    uint8_t *LSr, *LSc;  // mixed: slice stores of the L tiles (rows / columns as K-major rows)
    uint8_t *XSr, *XSc;  // mixed: slice stores of the L^{-1} tiles (diagonal: W_j)
    float *L32;          // mixed: FP32 tiles for the correction solves (L_ij, diagonal W_j)
    double *rp;          // mixed: residual partials per tile, C_ij a_j and C_ij^T a_i (2 x 128)
    int64_t n;
    int T;
    int ntasks;
    int kind;
    int mixed;
    double s2, scale, diag, tau2;
    dfl dscale, ds2, ddiag;  // mixed: double-float parameters
    int pad_;
};

constexpr int DAG_NSTAT = 10;  // task classes of the optional cycle counters

struct DagHdr {
    int next;   // ticket of the next task in the global list
    int abort;  // a wait timed out: every CTA stops
    int prof;   // count cycles per task class (diagnostics)
    int pad_[13];
    unsigned long long cyc[DAG_NSTAT];   // SM cycles inside tasks of the class
    unsigned long long wait[DAG_NSTAT];  // of which spent waiting for inputs
    unsigned long long cnt[DAG_NSTAT];   // tasks
    unsigned long long steps;            // tensor-core contraction steps (mixed)
    unsigned long long pad2_[7];
};

__host__ __device__ inline int dag_ntiles(int T) { return T * (T + 1) / 2; }
constexpr int DAG_EVALS = 4;   // refinement residual evaluations (mixed form)
constexpr int DAG_CHAIN = 2 * DAG_EVALS;  // chain stages: RES(e), CORR(e) ..., RES(last), FIN

__host__ __device__ inline int dag_ntasks(int T, int mixed) {
    if (!mixed) return dag_ntiles(T) + 1 + T * (T - 1) / 2 + dag_ntiles(T) + 1;
    return dag_ntiles(T) + 1 + T * (T - 1) / 2 + DAG_EVALS * dag_ntiles(T) + DAG_EVALS +
           dag_ntiles(T) + 1;
}

// Flags per problem.  FP64: L (ntiles), X (ntiles), solve, LG count.
// Mixed: L, X, solve, residual counts (DAG_EVALS), corrections
// (DAG_EVALS - 1), log-likelihood, LG count, converged.
__host__ __device__ inline int dag_nflags(int T, int mixed) {
    return 2 * dag_ntiles(T) + (mixed ? 3 + 2 * DAG_EVALS + 1 : 2);
}
__host__ __device__ inline int dag_solved_flag(int T) { return 2 * dag_ntiles(T); }
__host__ __device__ inline int dag_lg_flag(int T, int mixed) {
    return mixed ? 2 * dag_ntiles(T) + 2 * DAG_EVALS + 1 : 2 * dag_ntiles(T) + 1;
}

__host__ __device__ inline int tile_index(int T, int i, int j) {
    return j * T - j * (j - 1) / 2 + (i - j);
}

enum { DT_RES = 5, DT_CORR = 6, DT_FINLL = 7 };

__device__ inline void dag_decode_xt(int T, int q, int &i, int &k) {
    int kk = T - 2;
    while (q >= T - 1 - kk) {
        q -= T - 1 - kk;
        --kk;
    }
    i = kk + 1 + q;
    k = kk;
}

// Local task q of a problem with T tiles -> (type, i, k).  Order: CHOL by
// tile columns (diagonal first), SOLVE, TRTRI by columns from the right,
// LG by columns from the right, FINAL.  The mixed form threads its
// refinement chain (RES(e) for every lower tile, then CORR(e); after the last
// evaluation FINLL) through the TRTRI tasks in DAG_CHAIN segments, so that
// each stage of the chain sits well after the one it waits for.  A RES task
// returns its tile as i = row | (column << 16) and the evaluation in k.
__device__ inline int dag_decode(int T, int mixed, int q, int &i, int &k) {
    const int nc = dag_ntiles(T);
    if (q < nc) {
        int j = 0;
        while (q >= T - j) {
            q -= T - j;
            ++j;
        }
        i = j + q;
        k = j;
        return DT_CHOL;
    }
    q -= nc;
    if (q == 0) return DT_SOLVE;
    q -= 1;
    const int nt = T * (T - 1) / 2;
    if (!mixed) {
        if (q < nt) {
            dag_decode_xt(T, q, i, k);
            return DT_TRTRI;
        }
        q -= nt;
    } else {
        const int g = (nt + DAG_CHAIN - 1) / DAG_CHAIN;
        for (int s = 0; s < DAG_CHAIN; ++s) {
            const int lo = s * g;
            const int seg = lo >= nt ? 0 : (nt - lo < g ? nt - lo : g);
            if (q < seg) {
                dag_decode_xt(T, lo + q, i, k);
                return DT_TRTRI;
            }
            q -= seg;
            const int st = (s & 1) ? 1 : nc;  // RES(e): one task per tile; CORR(e) / FINLL: 1
            if (q < st) {
                k = s >> 1;  // evaluation
                if (s & 1) return s == DAG_CHAIN - 1 ? DT_FINLL : DT_CORR;
                int jj = 0;  // RES tile (i, jj) in column order; jj returned through k's pair
                while (q >= T - jj) {
                    q -= T - jj;
                    ++jj;
                }
                i = (jj + q) | (jj << 16);
                return DT_RES;
            }
            q -= st;
        }
    }
    if (q < nc) {
        int j = T - 1;
        while (q >= T - j) {
            q -= T - j;
            --j;
        }
        i = j + q;
        k = j;
        return DT_LG;
    }
    return DT_FINAL;
}

// Tensor-core (mixed) form: 128 x 128 tiles, three FP16 slices per operand.
// A slice store holds, per tile, the three slices as two 128-row x 64-column
// K-major atoms each in the 128-byte-swizzled layout of the tcgen05 shared-
// memory descriptors (row r at r * 128 bytes, 16-byte chunk c at chunk
// c ^ (r % 8)), so that a task copies it to shared memory verbatim; then the
// 128 row exponents.
constexpr int QB = 128;
constexpr int QS = 3;
constexpr int QATOM = QB * 128;                // 16 KB
constexpr int QSLICE = 2 * QATOM;              // 32 KB
constexpr int QOPER = QS * QSLICE;             // 96 KB
constexpr int QSTRIDE = QOPER + 1024;          // + exponents, 1 KB aligned
constexpr int QSCRATCH_DOUBLES = 7 * 64 * 64;  // per-CTA FP64 blocks of a diagonal tile

struct DagHdr;
int dag_tc_launch(int grid, DagHdr *hdr, const DagProb *probs, const int2 *list, int ntot,
                  const float2 *dftab, double *scratch, cudaStream_t s);

struct DagSmem {
    double sA[DB * DLD];
    double sB[DB * DLD];
    double tab[EXP_TAB];
    double2 xr[DB], xc[DB];
    double vr[DB], vc[DB];
    double red[4][DB];
    double dinv[DB];
    double lj[DB];
    double wred[3][8];
    int bad;
    int badcol;
    int task;
    int pad_;
    int ok[4];  // verdict of the last wait, spin cycles (as one 64-bit value at ok + 2)
};

// --------------------------------------------------------------------------
// synchronisation
// --------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait (thread 0, bounded) until *f >= target; every thread gets the verdict.
// okslot[0]: the verdict; okslot[2..3]: cycles spent spinning (accumulated
// for the optional counters).
static __device__ bool dag_wait(const int *f, int target, DagHdr *h, int64_t *info, int *okslot) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_gpu(f) < target) {
            const long long c0 = clock64();
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 0;; ++it) {
                if (ld_acquire_gpu(f) >= target) break;
                if (ld_relaxed_gpu(&h->abort)) {
                    ok = 0;
                    break;
                }
                __nanosleep(128);
                if (it >= DAG_WAIT_POLLS ||
                    ((it & 255) == 0 && globaltimer_ns() - t0 > DAG_WAIT_NS)) {
                    set_info(info, -1);
                    atomicExch(&h->abort, 1);
                    ok = 0;
                    break;
                }
            }
            *reinterpret_cast<long long *>(okslot + 2) += clock64() - c0;
        }
        *okslot = ok;
    }
    __syncthreads();
    return *okslot != 0;
}

// Optional per-class cycle counters around one task (thread 0).
__device__ __forceinline__ long long dag_stat_begin(const DagHdr *h, int *okslot) {
    if (!h->prof || threadIdx.x != 0) return 0;
    *reinterpret_cast<long long *>(okslot + 2) = 0;
    return clock64();
}
__device__ __forceinline__ void dag_stat_end(DagHdr *h, int cls, long long c0, const int *okslot) {
    if (!h->prof || threadIdx.x != 0) return;
    atomicAdd(&h->cyc[cls], (unsigned long long)(clock64() - c0));
    atomicAdd(&h->wait[cls], (unsigned long long)*reinterpret_cast<const long long *>(okslot + 2));
    atomicAdd(&h->cnt[cls], 1ull);
}

// All of the CTA's writes so far, then *f += 1 with release semantics.
__device__ __forceinline__ void dag_signal(int *f) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(f) : "memory");
    }
}

// --------------------------------------------------------------------------
// 64 x 64 FP64 tile products: acc (rows tx + 16a, columns ty + 16b of the
// tile, tx = tid % 16, ty = tid / 16) += sum_t opA(r, t) opB(t, c), or -=.
//   TA = 0: opA(r, t) = A[r + 64 t]     TA = 1: opA(r, t) = A[t + 64 r]
//   TB = 0: opB(t, c) = B[t + 64 c]     TB = 1: opB(t, c) = B[c + 64 t]
// Operands come through L2 (written by other CTAs in this launch).
// --------------------------------------------------------------------------
template <int TA>
__device__ __forceinline__ void stage_a(const double *A, double *sA) {
    for (int e = threadIdx.x; e < DB * DB; e += DAG_THREADS) {
        const double v = __ldcg(A + e);
        const int lo = e & (DB - 1), hi = e >> 6;
        if (TA == 0) sA[hi * DLD + lo] = v;  // r = lo, t = hi
        else sA[lo * DLD + hi] = v;          // t = lo, r = hi
    }
}

template <int TB>
__device__ __forceinline__ void stage_b(const double *B, double *sB) {
    for (int e = threadIdx.x; e < DB * DB; e += DAG_THREADS) {
        const double v = __ldcg(B + e);
        const int lo = e & (DB - 1), hi = e >> 6;
        if (TB == 0) sB[lo * DLD + hi] = v;  // t = lo, c = hi
        else sB[hi * DLD + lo] = v;          // c = lo, t = hi
    }
}

template <bool NEG>
__device__ __forceinline__ void mma_smem(double (&acc)[4][4], const double *sA, const double *sB) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 4
    for (int t = 0; t < DB; ++t) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = NEG ? -sA[t * DLD + tx + 16 * a] : sA[t * DLD + tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = sB[t * DLD + ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
}

template <int TA, int TB, bool NEG>
__device__ __forceinline__ void tile_mma(double (&acc)[4][4], const double *A, const double *B,
                                         DagSmem &sm) {
    __syncthreads();
    stage_a<TA>(A, sm.sA);
    stage_b<TB>(B, sm.sB);
    __syncthreads();
    mma_smem<NEG>(acc, sm.sA, sm.sB);
}

__device__ __forceinline__ void acc_zero(double (&acc)[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
}

// acc -> sA in the A-operand layout (sA[c * DLD + r] = acc(r, c)).
__device__ __forceinline__ void acc_to_sA(const double (&acc)[4][4], double *sA) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) sA[(ty + 16 * b) * DLD + tx + 16 * a] = acc[a][b];
}

__device__ __forceinline__ void acc_store(const double (&acc)[4][4], double *G) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) G[(tx + 16 * a) + DB * (ty + 16 * b)] = acc[a][b];
}

__device__ __forceinline__ double *tile_ptr(double *base, int T, int i, int j) {
    return base + (size_t)tile_index(T, i, j) * (DB * DB);
}

// --------------------------------------------------------------------------
// tasks
// --------------------------------------------------------------------------
// C_ij from the locations (identity on padded rows / columns).
static __device__ void fill_tile(const DagProb &P, int i, int j, double (&acc)[4][4], DagSmem &sm) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    __syncthreads();
    if (tid < DB) {
        const int64_t gi = (int64_t)i * DB + tid, gj = (int64_t)j * DB + tid;
        sm.xr[tid] = gi < P.n ? P.x[gi] : make_double2(0.0, 0.0);
        sm.xc[tid] = gj < P.n ? P.x[gj] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gi = (int64_t)i * DB + tx + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t gj = (int64_t)j * DB + ty + 16 * b;
            double v;
            if (gi >= P.n || gj >= P.n) v = (gi == gj) ? 1.0 : 0.0;
            else if (gi == gj) v = P.diag;
            else v = cov_offdiag_s(P.kind, P.s2, P.scale, pair_dist(sm.xr[tx + 16 * a], sm.xc[ty + 16 * b]), sm.tab);
            acc[a][b] = v;
        }
    }
}

// Cholesky of the 64 x 64 tile in sA (lower, unscaled-column form; a pivot <= 0 or
// NaN stops it and records the column), then L written to G, W = L^{-1} to
// Wg, and the tile's sum of log L_rr over rows < n to *logpart.
static __device__ void potrf_inv_tile(const DagProb &P, int j, double *G, double *Wg, double *logpart,
                               DagSmem &sm) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double *S = sm.sA;
    if (tid == 0) {
        sm.bad = 0;
        sm.badcol = 0;
    }
    __syncthreads();
    for (int jj = 0; jj < DB; ++jj) {
        const double *cj = S + jj * DLD;
        if (tid < DB) {
            const double d = cj[jj];
            if (!(d > 0.0)) {
                if (tid == 0) {
                    sm.bad = 1;
                    sm.badcol = jj;
                }
            } else {
                const double inv = 1.0 / d;
                if (tid == 0) sm.dinv[jj] = inv;
                if (tid > jj) sm.lj[tid] = cj[tid] * inv;
            }
        }
        __syncthreads();
        if (sm.bad) break;
        for (int c = jj + 1 + warp; c < DB; c += 8) {
            const double l = sm.lj[c];
            double *sc = S + c * DLD;
            for (int r = c + lane; r < DB; r += 32) sc[r] = fma(-cj[r], l, sc[r]);
        }
        __syncthreads();
    }
    if (sm.bad) {
        if (tid == 0) set_info(P.info, (int64_t)j * DB + sm.badcol + 1);
        return;
    }
    // L_rc = a_rc sqrt(1 / d_c); write L and keep it in S
    for (int e = tid; e < DB * DB; e += DAG_THREADS) {
        const int r = e & (DB - 1), c = e >> 6;
        const double v = (r >= c) ? S[c * DLD + r] * sqrt(sm.dinv[c]) : 0.0;
        S[c * DLD + r] = v;
        G[e] = v;
    }
    __syncthreads();
    if (tid < DB) {
        const double d = S[tid * DLD + tid];
        sm.lj[tid] = 1.0 / d;  // 1 / L_rr
        sm.vr[tid] = ((int64_t)j * DB + tid < P.n) ? log(d) : 0.0;
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
        if (r > c) S[c * DLD + r] *= sm.lj[r];
        sm.sB[c * DLD + r] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int l = DB - 1; l > 0; --l) {
        for (int e = tid; e < l * DB; e += DAG_THREADS) {
            const int c = e >> 6, r = e & (DB - 1);
            sm.sB[c * DLD + r] = fma(-sm.sB[l * DLD + r], S[c * DLD + l], sm.sB[c * DLD + r]);
        }
        __syncthreads();
    }
    for (int e = tid; e < DB * DB; e += DAG_THREADS) {
        const int r = e & (DB - 1), c = e >> 6;
        Wg[e] = (r >= c) ? sm.sB[c * DLD + r] * sm.lj[c] : 0.0;
    }
}

}  // namespace gp
