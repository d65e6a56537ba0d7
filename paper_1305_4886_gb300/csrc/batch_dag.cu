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
#include <mutex>
#include <stdlib.h>
#include <string.h>
#include <vector>

namespace gp {

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

// After an abort, every problem whose final task did not finish gets -1 (if
// it has no status yet) and NaN results; finished problems keep theirs.
__global__ void dag_finish_kernel(const DagHdr *h, const DagProb *probs, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !h->abort) return;
    const DagProb &d = probs[p];
    if (d.flag[dag_done_flag(d.T, d.mixed)] != 0) return;
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
    unsigned long long wait_ns;
    const int *unset;
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
        if (t == 0) {
            DagHdr *h = reinterpret_cast<DagHdr *>(hdr_raw);
            h->prof = s.prof;
            h->wait_ns = s.wait_ns;
            h->unset = s.unset;
        }
        if (t < EXP_TAB) tab[t] = s.tab[t];
        for (int q = t; q < DF_TAB; q += blockDim.x) dftab[q] = s.dftab[q];
    }
}


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
    const int r = round_of(j, N, R);
    const int64_t pos = roff[r] + poff[(int64_t)r * P + p] + (j - round_start(N, r, R));
    list[pos] = make_int2(p, j);
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
static size_t al1k(size_t x) { return (x + 1023) & ~size_t(1023); }

struct DagLayout {
    int P = 0, R = DAG_ROUNDS, maxN = 0, mixed = 0;
    int64_t ntot = 0;
    size_t flags = 0, flags_bytes = 0, probs = 0, tab = 0, dftab = 0, list = 0, poff = 0, rtot = 0,
           roff = 0, scratch = 0;
    std::vector<int> T, ntasks, order, tc;  // tc: the problem runs on tensor-core tiles
    std::vector<size_t> A, X, vec, part, flag, LSr, LSc, XSr, XSc, L32, rp;
    size_t total = 0;
};

// Bytes of one problem's own storage: FP64 tiles (64 x 64) or tensor-core
// tiles (128 x 128, slice stores of L and L^{-1} in both orientations, FP32
// tiles, residual partials).
static size_t prob_bytes(int64_t n, bool tc) {
    const int tb = tc ? QB : DB;
    const size_t T = (size_t)ceil_div(n, tb), nt = T * (T + 1) / 2, m = T * tb;
    size_t b = 0;
    if (!tc) {
        b += 2 * al256(sizeof(double) * nt * DB * DB);
    } else {
        b += 4 * al1k(nt * QSTRIDE) + al1k(sizeof(float) * nt * QB * QB) +
             al256(sizeof(double) * nt * 2 * QB);
    }
    b += al256(sizeof(double) * (tc ? 4 : 3) * m) + al256(sizeof(double) * (T + 3 * nt + (tc ? 4 : 0)));
    return b + 1024;  // alignment slack
}

// mixed: problems with n > fp64_max_n run on tensor-core tiles, the others
// on FP64 tiles in the same launch.  reserve: size every problem for the
// larger of its two layouts (so that any threshold fits the workspace).
static DagLayout dag_layout(int P, const int64_t *h_n, int mixed, int scratch_ctas,
                            int64_t fp64_max_n, bool reserve = false) {
    DagLayout L;
    L.P = P;
    L.mixed = mixed;
    L.T.resize(P);
    L.ntasks.resize(P);
    L.order.resize(P);
    L.tc.resize(P);
    for (int i = 0; i < P; ++i) L.order[i] = i;
    // largest problems first within every round
    std::stable_sort(L.order.begin(), L.order.end(), [&](int a, int b) { return h_n[a] > h_n[b]; });
    size_t nflag = 0;
    L.flag.resize(P);
    for (int s = 0; s < P; ++s) {
        const int64_t n = h_n[L.order[s]];
        const int tc = (mixed && n > fp64_max_n) ? 1 : 0;
        const int T = (int)ceil_div(n, tc ? QB : DB);
        L.tc[s] = tc;
        L.T[s] = T;
        L.ntasks[s] = dag_ntasks(T, tc);
        L.ntot += L.ntasks[s];
        L.maxN = std::max(L.maxN, L.ntasks[s]);
        L.flag[s] = nflag;
        nflag += (size_t)std::max(dag_nflags(T, tc),
                                  reserve ? dag_nflags((int)ceil_div(n, DB), 0) : 0);
    }
    if (reserve) {  // task list sized for the larger task count of either layout
        L.ntot = 0;
        for (int s = 0; s < P; ++s) {
            const int64_t n = h_n[L.order[s]];
            L.ntot += std::max(dag_ntasks((int)ceil_div(n, DB), 0),
                               mixed ? dag_ntasks((int)ceil_div(n, QB), 1) : 0);
        }
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
        const int64_t n = h_n[L.order[s]];
        const size_t start = off;
        const size_t nt = dag_ntiles(L.T[s]);
        const size_t m = (size_t)L.T[s] * (L.tc[s] ? QB : DB);
        off = al1k(off);
        if (!L.tc[s]) {
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
        off = al256(off + sizeof(double) * (L.tc[s] ? 4 : 3) * m);
        L.part[s] = off;
        off = al256(off + sizeof(double) * (L.T[s] + 3 * nt + (L.tc[s] ? 4 : 0)));
        if (reserve) {
            const size_t want = start + std::max(prob_bytes(n, false), mixed ? prob_bytes(n, true) : 0);
            off = std::max(off, want);
        }
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

// Largest problem on FP64 tiles in the mixed launch, per device (the tile
// policy; gp_batched_autotune measures it, gp_batched_set_tile_policy sets it).
static std::atomic<int64_t> g_fp64_max_n[64];
void dag_set_fp64_max_n(int64_t v) {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) g_fp64_max_n[dev].store(v);
}
int64_t dag_fp64_max_n() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    return g_fp64_max_n[dev].load();
}

// The wait limit of the batched launches and the testing aid that leaves one
// Cholesky tile flag of one problem unraised (process-wide settings).
static std::mutex g_wait_mu;
static uint64_t g_wait_ns = DAG_WAIT_NS;
static int g_unset_prob = -1;
static int64_t g_unset_i = 0, g_unset_j = 0;

int dag_set_wait_ns(uint64_t ns) {
    std::lock_guard<std::mutex> lk(g_wait_mu);
    g_wait_ns = ns;
    return GP_OK;
}

int dag_set_unset_tile(int prob, int64_t i, int64_t j) {
    if (prob >= 0 && (j < 0 || i < j)) return GP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_wait_mu);
    g_unset_prob = prob < 0 ? -1 : prob;
    g_unset_i = i;
    g_unset_j = j;
    return GP_OK;
}

size_t dag_workspace_bytes(int nprob, const int64_t *h_n, int mixed) {
    return dag_layout(nprob, h_n, mixed, mixed ? std::max(dag_tc_ctas(), 1) : 0, 0, true).total;
}

int dag_run(int nprob, const int64_t *h_n, const double *const *h_dx, const double *const *h_dy,
            const double *const *h_dmu, const KernParams *kps, int mixed, int64_t fp64_max_n,
            void *d_ws, size_t ws_bytes, double *d_out, double *d_grad, int64_t *d_info,
            cudaStream_t s) {
    if (nprob > 65535) return GP_ERR_INVALID;
    for (int i = 0; i < nprob; ++i)  // tile indices of a problem stay below 2^15 per side
        if (ceil_div(h_n[i], mixed ? QB : DB) > 8192) return GP_ERR_INVALID;
    const int tc_ctas = mixed ? dag_tc_ctas() : 0;
    if (mixed && tc_ctas < 1) return GP_ERR_CUDA;
    const DagLayout L = dag_layout(nprob, h_n, mixed, tc_ctas, fp64_max_n);
    if (L.total > ws_bytes) return GP_ERR_WORKSPACE;
    if (L.ntot >= (1ll << 31)) return GP_ERR_INVALID;
    char *base = static_cast<char *>(d_ws);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
    // set once per device; a race between host threads only repeats the
    // (idempotent) attribute call
    static std::atomic<bool> attr_set[64];
    if (!mixed && !attr_set[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(dag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(DagSmem)) != cudaSuccess)
            return GP_ERR_CUDA;
        attr_set[dev].store(true, std::memory_order_release);
    }
    if (cudaMemsetAsync(base + L.flags, 0, L.flags_bytes, s) != cudaSuccess) return GP_ERR_CUDA;
    DagHdr *hdr = reinterpret_cast<DagHdr *>(base + L.flags);
    int *flag0 = reinterpret_cast<int *>(base + L.flags + sizeof(DagHdr));
    DagProb *probs = reinterpret_cast<DagProb *>(base + L.probs);
    double *tab = reinterpret_cast<double *>(base + L.tab);
    float2 *dftab = reinterpret_cast<float2 *>(base + L.dftab);
    uint64_t wait_ns;
    const int *unset = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_wait_mu);
        wait_ns = g_wait_ns;
        if (g_unset_prob >= 0 && g_unset_prob < nprob) {
            int sidx = 0;
            while (L.order[sidx] != g_unset_prob) ++sidx;
            if (g_unset_i >= L.T[sidx]) return GP_ERR_INVALID;
            unset = flag0 + L.flag[sidx] + tile_index(L.T[sidx], (int)g_unset_i, (int)g_unset_j);
        }
    }
    // descriptors, in chunks of kernel parameters
    std::vector<DagSetup> chunks((nprob + DAG_SETUP_CHUNK - 1) / DAG_SETUP_CHUNK);
    for (int s0 = 0, c = 0; s0 < nprob; s0 += DAG_SETUP_CHUNK, ++c) {
        DagSetup &su = chunks[c];
        memset(&su, 0, sizeof(su));
        su.first = s0;
        su.count = std::min(DAG_SETUP_CHUNK, nprob - s0);
        su.prof = dag_profiling() ? 1 : 0;
        su.wait_ns = wait_ns;
        su.unset = unset;
        for (int q = 0; q < EXP_TAB; ++q) su.tab[q] = kps[0].tab[q];
        for (int q = 0; q < DF_TAB; ++q) su.dftab[q] = kps[0].kd.tab[q];
        for (int q = 0; q < su.count; ++q) {
            const int sidx = s0 + q, o = L.order[sidx];
            DagProb &d = su.p[q];
            d.x = reinterpret_cast<const double2 *>(h_dx[o]);
            d.y = h_dy[o];
            d.mu = h_dmu ? h_dmu[o] : nullptr;
            if (!L.tc[sidx]) {
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
            d.mixed = L.tc[sidx];
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
        GP_TRY(dag_tc_launch(grid, hdr, probs, list, (int)L.ntot, tab, dftab,
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

// --------------------------------------------------------------------------
// Host check of the ordering invariant (no device work): rebuild the merged
// global list of a batch as dag_plan_rounds / dag_plan_fill do, decode every
// task, list the flags it waits on (the waits of the task functions) and the
// tasks that raise them, and count the dependencies that are not earlier in
// the list (a correct plan has none: the launch cannot deadlock) and the
// list slots that are not exactly one task.
// --------------------------------------------------------------------------
int dag_plan_check(int nprob, const int64_t *h_n, int mixed, int64_t fp64_max_n, int64_t *h_ntasks,
                   int64_t *h_bad_order, int64_t *h_bad_slots) {
    if (nprob < 1 || nprob > 65535) return GP_ERR_INVALID;
    for (int i = 0; i < nprob; ++i)
        if (h_n[i] < 1 || ceil_div(h_n[i], mixed ? QB : DB) > 8192) return GP_ERR_INVALID;
    const DagLayout L = dag_layout(nprob, h_n, mixed, 1, fp64_max_n);
    const int R = L.R;
    // merged positions, as the device plan computes them
    std::vector<int64_t> rtot(R, 0), roff(R + 1, 0);
    std::vector<int64_t> poff((size_t)R * nprob, 0);
    for (int r = 0; r < R; ++r) {
        int64_t acc = 0;
        for (int p = 0; p < nprob; ++p) {
            const int64_t N = L.ntasks[p];
            poff[(size_t)r * nprob + p] = acc;
            acc += round_start(N, r + 1, R) - round_start(N, r, R);
        }
        rtot[r] = acc;
    }
    for (int r = 0; r < R; ++r) roff[r + 1] = roff[r] + rtot[r];
    std::vector<int64_t> base(nprob + 1, 0);
    for (int p = 0; p < nprob; ++p) base[p + 1] = base[p] + L.ntasks[p];
    std::vector<int64_t> pos(base[nprob], -1);
    std::vector<int> hits(L.ntot, 0);
    int64_t bad_slots = 0;
    for (int p = 0; p < nprob; ++p)
        for (int64_t j = 0; j < L.ntasks[p]; ++j) {
            const int64_t N = L.ntasks[p];
            const int r = round_of(j, N, R);
            const int64_t q = roff[r] + poff[(size_t)r * nprob + p] + (j - round_start(N, r, R));
            if (q < 0 || q >= L.ntot) {
                ++bad_slots;
                continue;
            }
            pos[base[p] + j] = q;
            ++hits[q];
        }
    for (int64_t q = 0; q < L.ntot; ++q)
        if (hits[q] != 1) ++bad_slots;
    // per problem: the producer of every flag (local task index) and the waits
    int64_t bad = 0;
    for (int p = 0; p < nprob; ++p) {
        const int T = L.T[p], tc = L.tc[p], N = L.ntasks[p];
        const int nt = dag_ntiles(T);
        std::vector<int> Lp(nt, -1), Xp(nt, -1);
        std::vector<std::vector<int>> resp(DAG_EVALS);
        std::vector<int> corrp(DAG_EVALS, -1), lgp;
        int solvep = -1, finp = -1;
        std::vector<int> type(N), ti(N), tk(N);
        for (int q = 0; q < N; ++q) {
            int i = 0, k = 0;
            const int t = dag_decode(T, tc, q, i, k);
            type[q] = t;
            ti[q] = i;
            tk[q] = k;
            switch (t) {
                case DT_CHOL:
                    Lp[tile_index(T, i, k)] = q;
                    if (i == k) Xp[tile_index(T, i, i)] = q;
                    break;
                case DT_TRTRI: Xp[tile_index(T, i, k)] = q; break;
                case DT_SOLVE: solvep = q; break;
                case DT_RES: resp[k].push_back(q); break;
                case DT_CORR: corrp[k] = q; break;
                case DT_FINLL: finp = q; break;
                case DT_LG: lgp.push_back(q); break;
                default: break;
            }
        }
        auto before = [&](int prod, int q) {
            if (prod < 0 || pos[base[p] + prod] >= pos[base[p] + q]) ++bad;
        };
        for (int q = 0; q < N; ++q) {
            const int i = ti[q], k = tk[q];
            switch (type[q]) {
                case DT_CHOL:
                    for (int m = 0; m < k; ++m) {
                        before(Lp[tile_index(T, i, m)], q);
                        before(Lp[tile_index(T, k, m)], q);
                    }
                    if (i > k) before(Lp[tile_index(T, k, k)], q);
                    break;
                case DT_SOLVE:
                    for (int a = 0; a < T; ++a)
                        for (int b = 0; b <= a; ++b) before(Lp[tile_index(T, a, b)], q);
                    break;
                case DT_TRTRI:
                    for (int m = k + 1; m <= i; ++m) {
                        before(Xp[tile_index(T, i, m)], q);
                        before(Lp[tile_index(T, m, k)], q);
                    }
                    before(Xp[tile_index(T, k, k)], q);
                    break;
                case DT_LG:
                    for (int m = i; m < T; ++m) {
                        before(Xp[tile_index(T, m, i)], q);
                        before(Xp[tile_index(T, m, k)], q);
                    }
                    before(tc ? finp : solvep, q);
                    break;
                case DT_RES:
                    before(k == 0 ? solvep : corrp[k - 1], q);
                    break;
                case DT_CORR:
                    if ((int)resp[k].size() != nt) ++bad;
                    for (int d : resp[k]) before(d, q);
                    break;
                case DT_FINLL:
                    if ((int)resp[DAG_EVALS - 1].size() != nt) ++bad;
                    for (int d : resp[DAG_EVALS - 1]) before(d, q);
                    break;
                default:  // FINAL
                    if ((int)lgp.size() != nt) ++bad;
                    for (int d : lgp) before(d, q);
                    break;
            }
        }
        for (int t = 0; t < nt; ++t)
            if (Lp[t] < 0 || Xp[t] < 0) ++bad;  // every tile has its producers
    }
    if (h_ntasks) *h_ntasks = L.ntot;
    if (h_bad_order) *h_bad_order = bad;
    if (h_bad_slots) *h_bad_slots = bad_slots;
    return GP_OK;
}

}  // namespace gp
