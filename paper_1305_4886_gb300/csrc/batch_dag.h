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
constexpr uint64_t DAG_WAIT_NS = 20ull * 1000 * 1000 * 1000;  // default limit of one wait: 20 s
constexpr uint32_t DAG_WAIT_POLLS = 1u << 30;  // a second guard on every wait (> 2 min of polls)

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
    int pad0_;
    unsigned long long wait_ns;  // limit of one dependency wait (host-set per call)
    const int *unset;            // testing aid: waits on this flag never see it raised
    int pad_[8];
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
// (DAG_EVALS - 1), log-likelihood, LG count, converged.  Both: a last flag
// raised when the problem's final task has written its results.
__host__ __device__ inline int dag_nflags(int T, int mixed) {
    return 2 * dag_ntiles(T) + (mixed ? 3 + 2 * DAG_EVALS + 1 : 2) + 1;
}
__host__ __device__ inline int dag_done_flag(int T, int mixed) { return dag_nflags(T, mixed) - 1; }
__host__ __device__ inline int dag_solved_flag(int T) { return 2 * dag_ntiles(T); }
__host__ __device__ inline int dag_lg_flag(int T, int mixed) {
    return mixed ? 2 * dag_ntiles(T) + 2 * DAG_EVALS + 1 : 2 * dag_ntiles(T) + 1;
}

__host__ __device__ inline int tile_index(int T, int i, int j) {
    return j * T - j * (j - 1) / 2 + (i - j);
}

enum { DT_RES = 5, DT_CORR = 6, DT_FINLL = 7 };

__host__ __device__ inline void dag_decode_xt(int T, int q, int &i, int &k) {
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
__host__ __device__ inline int dag_decode(int T, int mixed, int q, int &i, int &k) {
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

// First task of round r of R in a list of N tasks (the proportional merge).
__host__ __device__ inline int64_t round_start(int64_t N, int r, int R) { return (int64_t)r * N / R; }
// Round of local task j of a list of N tasks.
__host__ __device__ inline int round_of(int64_t j, int64_t N, int R) {
    return (int)(((j + 1) * (int64_t)R - 1) / N);
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
                  const double *tab, const float2 *dftab, double *scratch, cudaStream_t s);

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
    int ok[4];  // outcome of the last wait, spin cycles (as one 64-bit value at ok + 2)
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

// Wait (thread 0, bounded) until *f >= target; every thread gets the outcome.
// okslot[0]: the outcome; okslot[2..3]: cycles spent spinning (accumulated
// for the optional counters).
static __device__ bool dag_wait(const int *f, int target, DagHdr *h, int64_t *info, int *okslot) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        // the testing aid: a flag that counts as never raised
        if (f == h->unset) target = 0x7fffffff;
        if (ld_acquire_gpu(f) < target) {
            const long long c0 = clock64();
            const uint64_t t0 = globaltimer_ns();
            const uint64_t limit = h->wait_ns;
            for (uint32_t it = 0;; ++it) {
                if (ld_acquire_gpu(f) >= target) break;
                if (ld_relaxed_gpu(&h->abort)) {
                    ok = 0;
                    break;
                }
                __nanosleep(128);
                if (it >= DAG_WAIT_POLLS ||
                    ((it & 255) == 0 && globaltimer_ns() - t0 > limit)) {
                    set_info(info, -1);
                    atomicExch(&h->abort, 1);
                    ok = 0;
                    break;
                }
            }
            *reinterpret_cast<long long *>(okslot + 2) += clock64() - c0;
        }
        // the acquire, made cumulative for the CTA's other threads, whose
        // reads of the producer's tile follow the barrier below
        __threadfence();
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

// A problem's status (or any flag another CTA may set meanwhile) as ONE
// value for the whole CTA: every thread must take the same branch around
// the barriers that follow.  A barrier itself (all threads call it).
__device__ __forceinline__ bool dag_uniform(bool v) { return __syncthreads_or(v ? 1 : 0) != 0; }
__device__ __forceinline__ bool dag_failed(const DagProb &P) { return dag_uniform(failed(P.info)); }

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
        // a location that is not finite: d_info = -2 before any task can
        // read a tile built from it (the first status wins)
        if (!isfinite(sm.xr[tid].x) || !isfinite(sm.xr[tid].y) || !isfinite(sm.xc[tid].x) ||
            !isfinite(sm.xc[tid].y))
            set_info(P.info, -2);
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
    const int tid = threadIdx.x;
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
        // the trailing triangle flattened over all threads (every lane busy)
        const int ntri = (DB - 1 - jj) * (DB - jj) / 2;
        for (int e = tid; e < ntri; e += DAG_THREADS) {
            int r, c;
            tri_desc_entry(e, DB, r, c);
            S[c * DLD + r] = fma(-cj[r], sm.lj[c], S[c * DLD + r]);
        }
        __syncthreads();
    }
    if (sm.bad) {
        if (tid == 0) set_info(P.info, (int64_t)j * DB + sm.badcol + 1);
        return;
    }
    // L_rc = a_rc sqrt(1 / d_c), one square root per column; write L and keep it in S
    if (tid < DB) sm.dinv[tid] = sqrt(sm.dinv[tid]);
    __syncthreads();
    for (int e = tid; e < DB * DB; e += DAG_THREADS) {
        const int r = e & (DB - 1), c = e >> 6;
        const double v = (r >= c) ? S[c * DLD + r] * sm.dinv[c] : 0.0;
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
        // column l of Y is zero above row l: rows l.. only (exact zeros skipped)
        const int nr = DB - l;
        for (int e = tid; e < l * nr; e += DAG_THREADS) {
            const int c = e / nr, r = l + (e - c * nr);
            sm.sB[c * DLD + r] = fma(-sm.sB[l * DLD + r], S[c * DLD + l], sm.sB[c * DLD + r]);
        }
        __syncthreads();
    }
    for (int e = tid; e < DB * DB; e += DAG_THREADS) {
        const int r = e & (DB - 1), c = e >> 6;
        Wg[e] = (r >= c) ? sm.sB[c * DLD + r] * sm.lj[c] : 0.0;
    }
}

// --------------------------------------------------------------------------
// FP64 tile tasks (64 x 64 tiles, 256 threads; shared memory: DagSmem).
// They run in the FP64 launch and, for the problems given FP64 tiles, in the
// tensor-core launch.
// --------------------------------------------------------------------------
static __device__ bool task_chol(const DagProb &P, int i, int j, DagSmem &sm, DagHdr *h) {
    const int T = P.T;
    int *Lf = P.flag, *Xf = P.flag + dag_ntiles(T);
    const int tij = tile_index(T, i, j);
    if (!dag_failed(P)) {
        double acc[4][4];
        fill_tile(P, i, j, acc, sm);
        for (int k = 0; k < j; ++k) {
            if (!dag_wait(Lf + tile_index(T, i, k), 1, h, P.info, sm.ok)) return false;
            if (i != j && !dag_wait(Lf + tile_index(T, j, k), 1, h, P.info, sm.ok)) return false;
            tile_mma<0, 1, true>(acc, tile_ptr(P.A, T, i, k), tile_ptr(P.A, T, j, k), sm);
        }
        __syncthreads();
        acc_to_sA(acc, sm.sA);
        __syncthreads();
        if (i == j) {
            potrf_inv_tile(P, j, tile_ptr(P.A, T, j, j), tile_ptr(P.X, T, j, j), P.part + j, sm);
        } else {
            // L_ij = A'_ij W_j^T, W_j = X_jj
            if (!dag_wait(Lf + tile_index(T, j, j), 1, h, P.info, sm.ok)) return false;
            stage_b<1>(tile_ptr(P.X, T, j, j), sm.sB);
            __syncthreads();
            double l[4][4];
            acc_zero(l);
            mma_smem<false>(l, sm.sA, sm.sB);
            acc_store(l, tile_ptr(P.A, T, i, j));
        }
    }
    dag_signal(Lf + tij);
    if (i == j) dag_signal(Xf + tij);
    return true;
}

// Block sum of one value per thread (deterministic order); result in thread 0.
static __device__ double block_sum(double v, DagSmem &sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.wred[0][threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < DAG_THREADS / 32; ++w) s += sm.wred[0][w];
    return s;
}

static __device__ bool task_solve(const DagProb &P, DagSmem &sm, DagHdr *h) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * DB;
    int *Lf = P.flag;
    int *solved = P.flag + dag_solved_flag(T);
    double *r = P.vec, *v = P.vec + m, *al = P.vec + 2 * m;
    if (!dag_failed(P)) {
        for (int64_t e = tid; e < m; e += DAG_THREADS) {
            r[e] = e < P.n ? P.y[e] - (P.mu ? P.mu[e] : 0.0) : 0.0;
            if (!isfinite(r[e])) set_info(P.info, -2);
        }
        const int row = tid & (DB - 1), q = tid >> 6;
        // forward: v_i = W_i (r_i - sum_{j<i} L_ij v_j)
        for (int i = 0; i < T; ++i) {
            double s = 0.0;
            for (int j = 0; j < i; ++j) {
                if (!dag_wait(Lf + tile_index(T, i, j), 1, h, P.info, sm.ok)) return false;
                const double *L = tile_ptr(P.A, T, i, j);
                for (int c = q; c < DB; c += 4) s = fma(__ldcg(L + row + DB * c), v[(int64_t)j * DB + c], s);
            }
            if (!dag_wait(Lf + tile_index(T, i, i), 1, h, P.info, sm.ok)) return false;
            sm.red[q][row] = s;
            __syncthreads();
            if (tid < DB) sm.vr[tid] = r[(int64_t)i * DB + tid] - (sm.red[0][tid] + sm.red[1][tid] + sm.red[2][tid] + sm.red[3][tid]);
            __syncthreads();
            const double *W = tile_ptr(P.X, T, i, i);
            double t = 0.0;
            for (int c = q; c <= row; c += 4) t = fma(__ldcg(W + row + DB * c), sm.vr[c], t);
            sm.red[q][row] = t;
            __syncthreads();
            if (tid < DB) v[(int64_t)i * DB + tid] = sm.red[0][tid] + sm.red[1][tid] + sm.red[2][tid] + sm.red[3][tid];
            __syncthreads();
        }
        // logdet and q = v^T v
        double qs = 0.0;
        for (int64_t e = tid; e < P.n; e += DAG_THREADS) qs = fma(v[e], v[e], qs);
        const double quad = block_sum(qs, sm);
        // backward: alpha_i = W_i^T (v_i - sum_{j>i} L_ji^T alpha_j)
        for (int i = T - 1; i >= 0; --i) {
            double s = 0.0;
            for (int j = i + 1; j < T; ++j) {
                const double *L = tile_ptr(P.A, T, j, i);
                for (int c = q; c < DB; c += 4) s = fma(__ldcg(L + c + DB * row), al[(int64_t)j * DB + c], s);
            }
            sm.red[q][row] = s;
            __syncthreads();
            if (tid < DB) sm.vr[tid] = v[(int64_t)i * DB + tid] - (sm.red[0][tid] + sm.red[1][tid] + sm.red[2][tid] + sm.red[3][tid]);
            __syncthreads();
            const double *W = tile_ptr(P.X, T, i, i);
            double t = 0.0;
            for (int c = row + q; c < DB; c += 4) t = fma(__ldcg(W + c + DB * row), sm.vr[c], t);
            sm.red[q][row] = t;
            __syncthreads();
            if (tid < DB) al[(int64_t)i * DB + tid] = sm.red[0][tid] + sm.red[1][tid] + sm.red[2][tid] + sm.red[3][tid];
            __syncthreads();
        }
        if (tid == 0) {
            double ld = 0.0;
            for (int i = 0; i < T; ++i) ld += __ldcg(P.part + i);
            const double logdet = 2.0 * ld;
            const double LOG_2PI = 1.8378770664093454836;
            const bool bad = failed(P.info);
            P.out[0] = bad ? nan("") : -0.5 * logdet - 0.5 * quad - 0.5 * (double)P.n * LOG_2PI;
            P.out[1] = bad ? nan("") : logdet;
            P.out[2] = bad ? nan("") : quad;
            P.out[3] = bad ? nan("") : 0.0;
        }
    } else if (tid == 0) {
        P.out[0] = P.out[1] = P.out[2] = P.out[3] = nan("");
    }
    dag_signal(solved);
    return true;
}

static __device__ bool task_trtri(const DagProb &P, int i, int k, DagSmem &sm, DagHdr *h) {
    const int T = P.T;
    int *Lf = P.flag, *Xf = P.flag + dag_ntiles(T);
    if (!dag_failed(P)) {
        double acc[4][4];
        acc_zero(acc);
        for (int m = i; m > k; --m) {
            if (!dag_wait(Xf + tile_index(T, i, m), 1, h, P.info, sm.ok)) return false;
            if (!dag_wait(Lf + tile_index(T, m, k), 1, h, P.info, sm.ok)) return false;
            tile_mma<0, 0, false>(acc, tile_ptr(P.X, T, i, m), tile_ptr(P.A, T, m, k), sm);
        }
        if (!dag_wait(Xf + tile_index(T, k, k), 1, h, P.info, sm.ok)) return false;
        __syncthreads();
        acc_to_sA(acc, sm.sA);
        stage_b<0>(tile_ptr(P.X, T, k, k), sm.sB);
        __syncthreads();
        double x[4][4];
        acc_zero(x);
        mma_smem<true>(x, sm.sA, sm.sB);
        acc_store(x, tile_ptr(P.X, T, i, k));
    }
    dag_signal(Xf + tile_index(T, i, k));
    return true;
}

static __device__ bool task_lg(const DagProb &P, int i, int j, DagSmem &sm, DagHdr *h) {
    const int T = P.T, tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    int *Xf = P.flag + dag_ntiles(T);
    int *solved = P.flag + dag_solved_flag(T);
    int *lgc = P.flag + dag_lg_flag(T, 0);
    const int64_t m = (int64_t)T * DB;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (!dag_failed(P)) {
        double w[4][4];
        acc_zero(w);
        for (int mm = i; mm < T; ++mm) {
            if (!dag_wait(Xf + tile_index(T, mm, i), 1, h, P.info, sm.ok)) return false;
            if (!dag_wait(Xf + tile_index(T, mm, j), 1, h, P.info, sm.ok)) return false;
            tile_mma<1, 0, false>(w, tile_ptr(P.X, T, mm, i), tile_ptr(P.X, T, mm, j), sm);
        }
        if (!dag_wait(solved, 1, h, P.info, sm.ok)) return false;
        const double *al = P.vec + 2 * m;
        if (tid < DB) {
            const int64_t gi = (int64_t)i * DB + tid, gj = (int64_t)j * DB + tid;
            sm.xr[tid] = gi < P.n ? P.x[gi] : make_double2(0.0, 0.0);
            sm.xc[tid] = gj < P.n ? P.x[gj] : make_double2(0.0, 0.0);
            sm.vr[tid] = __ldcg(al + gi);
            sm.vc[tid] = __ldcg(al + gj);
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t gi = (int64_t)i * DB + tx + 16 * a;
            if (gi >= P.n) continue;
            const double ai = sm.vr[tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t gj = (int64_t)j * DB + ty + 16 * b;
                if (gj >= P.n || gj > gi) continue;
                if (gj == gi) {
                    const double cb = 0.5 * (ai * ai - w[a][b]);
                    g0 = fma(cb, P.s2, g0);
                    g2 = fma(cb, P.tau2, g2);
                } else {
                    const double cb2 = fma(ai, sm.vc[ty + 16 * b], -w[a][b]);
                    double cv, dr;
                    cov_and_dlogrho_s(P.kind, P.s2, P.scale,
                                      pair_dist(sm.xr[tx + 16 * a], sm.xc[ty + 16 * b]), cv, dr,
                                      sm.tab);
                    g0 = fma(cb2, cv, g0);
                    g1 = fma(cb2, dr, g1);
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
        g1 += __shfl_xor_sync(0xffffffffu, g1, o);
        g2 += __shfl_xor_sync(0xffffffffu, g2, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) {
        sm.wred[0][tid >> 5] = g0;
        sm.wred[1][tid >> 5] = g1;
        sm.wred[2][tid >> 5] = g2;
    }
    __syncthreads();
    if (tid < 3) {
        double s = 0.0;
        for (int w8 = 0; w8 < DAG_THREADS / 32; ++w8) s += sm.wred[tid][w8];
        P.part[T + 3 * tile_index(T, i, j) + tid] = s;
    }
    dag_signal(lgc);
    return true;
}

static __device__ bool task_final(const DagProb &P, DagSmem &sm, DagHdr *h) {
    const int T = P.T, tid = threadIdx.x;
    int *lgc = P.flag + dag_lg_flag(T, 0);
    const int nt = dag_ntiles(T);
    if (!dag_wait(lgc, nt, h, P.info, sm.ok)) return false;
    const bool bad = dag_failed(P);
    // Neumaier sums per thread, then in thread order
    double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
    for (int t = tid; t < nt; t += DAG_THREADS)
        for (int q = 0; q < 3; ++q) {
            const double x = __ldcg(P.part + T + 3 * t + q), u = s[q] + x;
            c[q] += (fabs(s[q]) >= fabs(x)) ? (s[q] - u) + x : (x - u) + s[q];
            s[q] = u;
        }
    __syncthreads();
    // 256 partials -> shared memory (sB as scratch)
    for (int q = 0; q < 3; ++q) sm.sB[q * DAG_THREADS + tid] = s[q] + c[q];
    __syncthreads();
    if (tid < 3) {
        double S = 0.0, C = 0.0;
        for (int t = 0; t < DAG_THREADS; ++t) {
            const double x = sm.sB[tid * DAG_THREADS + t], u = S + x;
            C += (fabs(S) >= fabs(x)) ? (S - u) + x : (x - u) + S;
            S = u;
        }
        P.grad[tid] = bad ? nan("") : S + C;
    }
    dag_signal(P.flag + dag_done_flag(T, 0));
    return true;
}

}  // namespace gp
