// batch_dag.cu -- many independent log-likelihood + gradient evaluations of
// uneven n as ONE persistent launch over a task graph (FP64 form).
//
// Every problem is cut into 64 x 64 tiles (n padded to a tile multiple with
// identity rows) and its whole evaluation into owner-computes tile tasks, in
// a topological order of the problem's own dependency graph:
//
//   CHOL(i, j), i >= j   left-looking tiled Cholesky (Sec. 2.1, by tiles):
//                        A'_ij = C_ij - sum_{k<j} L_ik L_jk^T, with C_ij
//                        recomputed from the locations (the fill is fused);
//                        i == j: L_jj = chol(A'_jj) in shared memory, plus
//                        W_j = L_jj^{-1} and sum_r log (L_jj)_rr;
//                        i > j: L_ij = A'_ij W_j^T (the panel solve).
//   SOLVE                v = L^{-1} r, logdet, q = v^T v, alpha = L^{-T} v
//                        (Sec. 2.2.2), by tile rows with W_i on the diagonal.
//   TRTRI(i, k), i > k   X = L^{-1} by tiles: X_kk = W_k and
//                        X_ik = -(sum_{m=k+1}^{i} X_im L_mk) W_k.
//   LG(i, j), i >= j     W_ij = sum_{m>=i} X_mi^T X_mj (a tile of C^{-1} =
//                        X^T X), contracted at once with alpha and with
//                        C_ij, dC_ij/dlog rho recomputed from the locations:
//                        the tile's share of the gradient (the adjoint
//                        1/2 (alpha alpha^T - C^{-1}) against dC/dtheta).
//   FINAL                the gradient from the tile shares (compensated).
//
// Each task writes its own tile once and raises a flag; a task that needs a
// tile waits for that flag just before it reads the tile (a bounded spin by
// one thread with acquire loads; tiles are then read through L2).  The
// problems' lists are merged into one global list in proportion to their
// lengths (round r of R takes, from every problem, the tasks whose position
// falls in [r/R, (r+1)/R) of its list), so that all problems advance
// together and a problem's dependent tasks sit far apart in the list.  The
// persistent CTAs take tasks from the list in order with one atomic ticket.
// Since every task waits only on tasks earlier in the list, the earliest
// task in progress always has its inputs: the schedule cannot deadlock,
// whatever the number of resident CTAs.  A wait that runs past its limit
// sets the problem's d_info to -1 and stops every CTA.
#include "batch_dag.h"

#include <algorithm>
#include <atomic>
#include <stdlib.h>
#include <string.h>
#include <vector>

namespace gp {

__device__ bool task_chol(const DagProb &P, int i, int j, DagSmem &sm, DagHdr *h) {
    const int T = P.T;
    int *Lf = P.flag, *Xf = P.flag + dag_ntiles(T);
    const int tij = tile_index(T, i, j);
    if (!failed(P.info)) {
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
__device__ double block_sum(double v, DagSmem &sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.wred[0][threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < DAG_THREADS / 32; ++w) s += sm.wred[0][w];
    return s;
}

__device__ bool task_solve(const DagProb &P, DagSmem &sm, DagHdr *h) {
    const int T = P.T, tid = threadIdx.x;
    const int64_t m = (int64_t)T * DB;
    int *Lf = P.flag;
    int *solved = P.flag + dag_solved_flag(T);
    double *r = P.vec, *v = P.vec + m, *al = P.vec + 2 * m;
    if (!failed(P.info)) {
        for (int64_t e = tid; e < m; e += DAG_THREADS)
            r[e] = e < P.n ? P.y[e] - (P.mu ? P.mu[e] : 0.0) : 0.0;
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

__device__ bool task_trtri(const DagProb &P, int i, int k, DagSmem &sm, DagHdr *h) {
    const int T = P.T;
    int *Lf = P.flag, *Xf = P.flag + dag_ntiles(T);
    if (!failed(P.info)) {
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

__device__ bool task_lg(const DagProb &P, int i, int j, DagSmem &sm, DagHdr *h) {
    const int T = P.T, tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    int *Xf = P.flag + dag_ntiles(T);
    int *solved = P.flag + dag_solved_flag(T);
    int *lgc = P.flag + dag_lg_flag(T, 0);
    const int64_t m = (int64_t)T * DB;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (!failed(P.info)) {
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

__device__ bool task_final(const DagProb &P, DagSmem &sm, DagHdr *h) {
    const int T = P.T, tid = threadIdx.x;
    int *lgc = P.flag + dag_lg_flag(T, 0);
    const int nt = dag_ntiles(T);
    if (!dag_wait(lgc, nt, h, P.info, sm.ok)) return false;
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
        P.grad[tid] = failed(P.info) ? nan("") : S + C;
    }
    return true;
}

__global__ void __launch_bounds__(DAG_THREADS, 2)
    dag_kernel(DagHdr *h, const DagProb *probs, const int2 *list, int ntot, const double *tab) {
    extern __shared__ __align__(16) unsigned char dag_smem_raw[];
    DagSmem &sm = *reinterpret_cast<DagSmem *>(dag_smem_raw);
    const int tid = threadIdx.x;
    if (tid < EXP_TAB) sm.tab[tid] = tab[tid];
    __syncthreads();
    for (;;) {
        if (tid == 0) sm.task = ld_relaxed_gpu(&h->abort) ? ntot : atomicAdd(&h->next, 1);
        __syncthreads();
        const int t = sm.task;
        __syncthreads();
        if (t >= ntot) break;
        const int2 e = list[t];
        const DagProb &P = probs[e.x];
        int i = 0, k = 0;
        const int type = dag_decode(P.T, 0, e.y, i, k);
        const long long c0 = dag_stat_begin(h, sm.ok);
        bool ok = true;
        switch (type) {
            case DT_CHOL: ok = task_chol(P, i, k, sm, h); break;
            case DT_SOLVE: ok = task_solve(P, sm, h); break;
            case DT_TRTRI: ok = task_trtri(P, i, k, sm, h); break;
            case DT_LG: ok = task_lg(P, i, k, sm, h); break;
            default: ok = task_final(P, sm, h); break;
        }
        dag_stat_end(h, (type == DT_CHOL && i == k) ? 8 : type, c0, sm.ok);
        if (!ok) break;
    }
}

// After an abort, every problem still without a status gets -1 and NaN.
__global__ void dag_finish_kernel(const DagHdr *h, const DagProb *probs, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !h->abort) return;
    const DagProb &d = probs[p];
    if (*d.info == 0) *d.info = -1;
    for (int q = 0; q < 4; ++q) d.out[q] = nan("");
    for (int q = 0; q < 3; ++q) d.grad[q] = nan("");
}

// --------------------------------------------------------------------------
// set-up: descriptors through kernel parameters (graph-capturable, no host
// staging buffer), then the proportional merge of the task lists.
// --------------------------------------------------------------------------
constexpr int DAG_SETUP_CHUNK = 128;
struct DagSetup {
    int first, count, prof, pad_;
    double tab[EXP_TAB];
    float2 dftab[DF_TAB];
    DagProb p[DAG_SETUP_CHUNK];
};
static_assert(sizeof(DagSetup) <= 32000, "descriptor chunk exceeds the kernel-parameter limit");

__global__ void dag_setup_kernel(const __grid_constant__ DagSetup s, DagProb *probs, double *tab,
                                 float2 *dftab, void *hdr_raw) {
    const int t = threadIdx.x;
    if (t < s.count) {
        probs[s.first + t] = s.p[t];
        *s.p[t].info = 0;
    }
    if (s.first == 0) {
        if (t == 0) reinterpret_cast<DagHdr *>(hdr_raw)->prof = s.prof;
        if (t < EXP_TAB) tab[t] = s.tab[t];
        for (int q = t; q < DF_TAB; q += blockDim.x) dftab[q] = s.dftab[q];
    }
}

__device__ __forceinline__ int64_t round_start(int64_t N, int r, int R) { return (int64_t)r * N / R; }

// One CTA per round: exclusive scan over problems of their task counts in
// the round; poff[r * P + p], rtot[r].
__global__ void __launch_bounds__(256) dag_plan_rounds(const DagProb *probs, int P, int R, int *poff,
                                                       int *rtot) {
    __shared__ int ws[8];
    __shared__ int carry;
    const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < P; base += 256) {
        const int p = base + tid;
        int c = 0;
        if (p < P) {
            const int64_t N = probs[p].ntasks;
            c = (int)(round_start(N, r + 1, R) - round_start(N, r, R));
        }
        int x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        int pre = carry;
        for (int q = 0; q < w; ++q) pre += ws[q];
        if (p < P) poff[(int64_t)r * P + p] = pre + x - c;
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int q = 0; q < 8; ++q) tot += ws[q];
            carry += tot;
        }
        __syncthreads();
    }
    if (tid == 0) rtot[r] = carry;
}

__global__ void dag_plan_scan(const int *rtot, int R, int *roff) {
    if (threadIdx.x == 0) {
        int s = 0;
        for (int r = 0; r < R; ++r) {
            roff[r] = s;
            s += rtot[r];
        }
        roff[R] = s;
    }
}

__global__ void dag_plan_fill(const DagProb *probs, int P, int R, const int *poff, const int *roff,
                              int2 *list) {
    const int p = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = probs[p].ntasks;
    if (j >= N) return;
    const int r = (int)(((int64_t)(j + 1) * R - 1) / N);
    const int64_t pos = roff[r] + poff[(int64_t)r * P + p] + (j - round_start(N, r, R));
    list[pos] = make_int2(p, j);
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
static size_t al1k(size_t x) { return (x + 1023) & ~size_t(1023); }

struct DagLayout {
    int P = 0, R = DAG_ROUNDS, maxN = 0, mixed = 0, tb = DB;
    int64_t ntot = 0;
    size_t flags = 0, flags_bytes = 0, probs = 0, tab = 0, dftab = 0, list = 0, poff = 0, rtot = 0,
           roff = 0, scratch = 0;
    std::vector<int> T, ntasks, order;
    std::vector<size_t> A, X, vec, part, flag, LSr, LSc, XSr, XSc, L32, rp;
    size_t total = 0;
};

static DagLayout dag_layout(int P, const int64_t *h_n, int mixed, int scratch_ctas) {
    DagLayout L;
    L.P = P;
    L.mixed = mixed;
    L.tb = mixed ? QB : DB;
    L.T.resize(P);
    L.ntasks.resize(P);
    L.order.resize(P);
    for (int i = 0; i < P; ++i) L.order[i] = i;
    // largest problems first within every round
    std::stable_sort(L.order.begin(), L.order.end(), [&](int a, int b) { return h_n[a] > h_n[b]; });
    size_t nflag = 0;
    L.flag.resize(P);
    for (int s = 0; s < P; ++s) {
        const int T = (int)ceil_div(h_n[L.order[s]], L.tb);
        L.T[s] = T;
        L.ntasks[s] = dag_ntasks(T, mixed);
        L.ntot += L.ntasks[s];
        L.maxN = std::max(L.maxN, L.ntasks[s]);
        L.flag[s] = nflag;
        nflag += (size_t)dag_nflags(T, mixed);
    }
    size_t off = 0;
    L.flags = off;
    L.flags_bytes = sizeof(DagHdr) + sizeof(int) * nflag;
    off = al256(off + L.flags_bytes);
    L.probs = off;
    off = al256(off + sizeof(DagProb) * P);
    L.tab = off;
    off = al256(off + sizeof(double) * EXP_TAB);
    L.dftab = off;
    off = al256(off + sizeof(float2) * DF_TAB);
    L.list = off;
    off = al256(off + sizeof(int2) * L.ntot);
    L.poff = off;
    off = al256(off + sizeof(int) * (size_t)L.R * P);
    L.rtot = off;
    off = al256(off + sizeof(int) * L.R);
    L.roff = off;
    off = al1k(off + sizeof(int) * (L.R + 1));
    L.scratch = off;
    if (mixed) off = al1k(off + (size_t)scratch_ctas * QSCRATCH_DOUBLES * sizeof(double));
    for (auto *v : {&L.A, &L.X, &L.vec, &L.part, &L.LSr, &L.LSc, &L.XSr, &L.XSc, &L.L32, &L.rp})
        v->assign(P, 0);
    for (int s = 0; s < P; ++s) {
        const size_t nt = dag_ntiles(L.T[s]);
        const size_t m = (size_t)L.T[s] * L.tb;
        if (!mixed) {
            L.A[s] = off;
            off = al256(off + sizeof(double) * nt * DB * DB);
            L.X[s] = off;
            off = al256(off + sizeof(double) * nt * DB * DB);
        } else {
            for (auto *v : {&L.LSr, &L.LSc, &L.XSr, &L.XSc}) {
                (*v)[s] = off;
                off = al1k(off + nt * QSTRIDE);
            }
            L.L32[s] = off;
            off = al1k(off + sizeof(float) * nt * QB * QB);
            L.rp[s] = off;
            off = al256(off + sizeof(double) * nt * 2 * QB);
        }
        L.vec[s] = off;
        off = al256(off + sizeof(double) * (mixed ? 4 : 3) * m);
        L.part[s] = off;
        off = al256(off + sizeof(double) * (L.T[s] + 3 * nt + (mixed ? 4 : 0)));
    }
    L.total = off;
    return L;
}

// CTAs of the mixed launch (each owns a slice of FP64 scratch in the workspace).
static int dag_tc_ctas() {
    static int n = 0;
    if (!n) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        n = sms;  // one CTA per SM (the CTA takes most of the shared memory)
    }
    return n;
}

// Per-class cycle counters of the batched launches (diagnostics): off unless
// turned on by dag_set_profile or GP_DAG_PROFILE=1.
static std::atomic<int> g_dag_prof{-1};
void dag_set_profile(int on) { g_dag_prof.store(on ? 1 : 0); }
static bool dag_profiling() {
    int v = g_dag_prof.load();
    if (v < 0) {
        const char *e = getenv("GP_DAG_PROFILE");
        v = (e && e[0] == '1') ? 1 : 0;
        g_dag_prof.store(v);
    }
    return v == 1;
}

size_t dag_workspace_bytes(int nprob, const int64_t *h_n, int mixed) {
    return dag_layout(nprob, h_n, mixed, mixed ? std::max(dag_tc_ctas(), 1) : 0).total;
}

int dag_run(int nprob, const int64_t *h_n, const double *const *h_dx, const double *const *h_dy,
            const double *const *h_dmu, const KernParams *kps, int mixed, void *d_ws,
            size_t ws_bytes, double *d_out, double *d_grad, int64_t *d_info, cudaStream_t s) {
    if (nprob > 65535) return GP_ERR_INVALID;
    for (int i = 0; i < nprob; ++i)  // tile indices of a problem stay below 2^15 per side
        if (ceil_div(h_n[i], mixed ? QB : DB) > 8192) return GP_ERR_INVALID;
    const int tc_ctas = mixed ? dag_tc_ctas() : 0;
    if (mixed && tc_ctas < 1) return GP_ERR_CUDA;
    const DagLayout L = dag_layout(nprob, h_n, mixed, tc_ctas);
    if (L.total > ws_bytes) return GP_ERR_WORKSPACE;
    if (L.ntot >= (1ll << 31)) return GP_ERR_INVALID;
    char *base = static_cast<char *>(d_ws);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
    static bool attr_set[64] = {};
    if (!mixed && !attr_set[dev]) {
        if (cudaFuncSetAttribute(dag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(DagSmem)) != cudaSuccess)
            return GP_ERR_CUDA;
        attr_set[dev] = true;
    }
    if (cudaMemsetAsync(base + L.flags, 0, L.flags_bytes, s) != cudaSuccess) return GP_ERR_CUDA;
    DagHdr *hdr = reinterpret_cast<DagHdr *>(base + L.flags);
    int *flag0 = reinterpret_cast<int *>(base + L.flags + sizeof(DagHdr));
    DagProb *probs = reinterpret_cast<DagProb *>(base + L.probs);
    double *tab = reinterpret_cast<double *>(base + L.tab);
    float2 *dftab = reinterpret_cast<float2 *>(base + L.dftab);
    // descriptors, in chunks of kernel parameters
    std::vector<DagSetup> chunks((nprob + DAG_SETUP_CHUNK - 1) / DAG_SETUP_CHUNK);
    for (int s0 = 0, c = 0; s0 < nprob; s0 += DAG_SETUP_CHUNK, ++c) {
        DagSetup &su = chunks[c];
        memset(&su, 0, sizeof(su));
        su.first = s0;
        su.count = std::min(DAG_SETUP_CHUNK, nprob - s0);
        su.prof = dag_profiling() ? 1 : 0;
        for (int q = 0; q < EXP_TAB; ++q) su.tab[q] = kps[0].tab[q];
        for (int q = 0; q < DF_TAB; ++q) su.dftab[q] = kps[0].kd.tab[q];
        for (int q = 0; q < su.count; ++q) {
            const int sidx = s0 + q, o = L.order[sidx];
            DagProb &d = su.p[q];
            d.x = reinterpret_cast<const double2 *>(h_dx[o]);
            d.y = h_dy[o];
            d.mu = h_dmu ? h_dmu[o] : nullptr;
            if (!mixed) {
                d.A = reinterpret_cast<double *>(base + L.A[sidx]);
                d.X = reinterpret_cast<double *>(base + L.X[sidx]);
            } else {
                d.LSr = reinterpret_cast<uint8_t *>(base + L.LSr[sidx]);
                d.LSc = reinterpret_cast<uint8_t *>(base + L.LSc[sidx]);
                d.XSr = reinterpret_cast<uint8_t *>(base + L.XSr[sidx]);
                d.XSc = reinterpret_cast<uint8_t *>(base + L.XSc[sidx]);
                d.L32 = reinterpret_cast<float *>(base + L.L32[sidx]);
                d.rp = reinterpret_cast<double *>(base + L.rp[sidx]);
            }
            d.vec = reinterpret_cast<double *>(base + L.vec[sidx]);
            d.part = reinterpret_cast<double *>(base + L.part[sidx]);
            d.flag = flag0 + L.flag[sidx];
            d.out = d_out + 4 * (size_t)o;
            d.grad = d_grad + 3 * (size_t)o;
            d.info = d_info + o;
            d.n = h_n[o];
            d.T = L.T[sidx];
            d.ntasks = L.ntasks[sidx];
            d.kind = kps[o].kind;
            d.mixed = mixed;
            d.s2 = kps[o].s2;
            d.scale = kps[o].scale;
            d.diag = kps[o].diag;
            d.tau2 = kps[o].tau2;
            d.dscale = kps[o].kd.scale;
            d.ds2 = kps[o].kd.s2;
            d.ddiag = kps[o].kd.diag;
        }
        dag_setup_kernel<<<1, DAG_SETUP_CHUNK, 0, s>>>(su, probs, tab, dftab, hdr);
        GP_LAUNCH_CHECK();
    }
    int *poff = reinterpret_cast<int *>(base + L.poff);
    int *rtot = reinterpret_cast<int *>(base + L.rtot);
    int *roff = reinterpret_cast<int *>(base + L.roff);
    int2 *list = reinterpret_cast<int2 *>(base + L.list);
    dag_plan_rounds<<<L.R, 256, 0, s>>>(probs, nprob, L.R, poff, rtot);
    GP_LAUNCH_CHECK();
    dag_plan_scan<<<1, 32, 0, s>>>(rtot, L.R, roff);
    GP_LAUNCH_CHECK();
    dag_plan_fill<<<dim3((unsigned)ceil_div(L.maxN, 256), (unsigned)nprob), 256, 0, s>>>(
        probs, nprob, L.R, poff, roff, list);
    GP_LAUNCH_CHECK();
    if (!mixed) {
        int sms = 0, occ = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dag_kernel, DAG_THREADS,
                                                          sizeof(DagSmem)) != cudaSuccess)
            return GP_ERR_CUDA;
        if (occ < 1) return GP_ERR_CUDA;
        const int grid = (int)std::min<int64_t>((int64_t)sms * occ, L.ntot);
        dag_kernel<<<grid, DAG_THREADS, sizeof(DagSmem), s>>>(hdr, probs, list, (int)L.ntot, tab);
        GP_LAUNCH_CHECK();
    } else {
        const int grid = (int)std::min<int64_t>(tc_ctas, L.ntot);
        GP_TRY(dag_tc_launch(grid, hdr, probs, list, (int)L.ntot, dftab,
                             reinterpret_cast<double *>(base + L.scratch), s));
    }
    dag_finish_kernel<<<(unsigned)ceil_div(nprob, 128), 128, 0, s>>>(hdr, probs, nprob);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

// Copy the counters of the last batched launch on this workspace (after a
// synchronisation): per class cycles, wait cycles, tasks; then steps.
int dag_stats(const void *d_ws, unsigned long long *h_out) {
    DagHdr hd;
    if (cudaMemcpy(&hd, d_ws, sizeof(hd), cudaMemcpyDeviceToHost) != cudaSuccess) return GP_ERR_CUDA;
    for (int q = 0; q < DAG_NSTAT; ++q) {
        h_out[q] = hd.cyc[q];
        h_out[DAG_NSTAT + q] = hd.wait[q];
        h_out[2 * DAG_NSTAT + q] = hd.cnt[q];
    }
    h_out[3 * DAG_NSTAT] = hd.steps;
    return GP_OK;
}

}  // namespace gp
