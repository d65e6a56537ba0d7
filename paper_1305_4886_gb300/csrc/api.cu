// api.cu -- the extern "C" entry points of libgp (declared in include/gp.h):
// argument checks, workspace carving and the launch sequence of each step.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "kern.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

namespace gp {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static bool params_ok(const gp_params *p) {
    if (!p) return false;
    if (p->kernel < GP_KERNEL_EXP || p->kernel > GP_KERNEL_MATERN52) return false;
    if (!(p->sigma2 > 0.0) || !(p->rho > 0.0) || !(p->tau2 >= 0.0)) return false;
    if (!isfinite(p->sigma2) || !isfinite(p->rho) || !isfinite(p->tau2)) return false;
    return true;
}

static bool precision_ok(int p) { return p == GP_FP64 || p == GP_MIXED_F16 || p == GP_EMU_FP64; }

int64_t padded(int64_t n) { return n < 1 ? 0 : round_up(n, PAD); }

// BF16 slices per FP64 operand: 3 in the mixed form (6 slice products), 5
// integer slices in the FP64-grade emulation (15 products).
static int slices_of(int precision) { return precision == GP_EMU_FP64 ? 5 : 3; }
constexpr int REFINE_EVALS = 4;      // residual evaluations of the mixed refinement
constexpr double REFINE_TOL = 1e-11; // ||r - C alpha|| / ||r|| target

// Workspace of the factorisation (beyond the matrix itself).
static size_t chol_ws_bytes(int64_t np, int precision) {
    if (precision == GP_FP64) return 0;
    return chol_mixed_ws_bytes(np, slices_of(precision));
}

struct LoglikWs {
    double *A = nullptr;      // n_p x n_p matrix (C, then L)
    double *r = nullptr;      // y - mu (n_p)
    double *v = nullptr;      // forward solve / alpha (n_p)
    double *acc = nullptr;    // C alpha (n_p)
    double *s = nullptr;      // refinement residual / correction (n_p)
    double *stats = nullptr;  // [0] refinement residual ratio
    int *conv = nullptr;      // refinement converged flag
    int *tsync = nullptr;     // ticket + flags of the single-launch solves
    double *winv = nullptr;   // tensor-core forms with gradient: the factorisation's
                              // diagonal-block inverses, reused by the inverse
    void *chol = nullptr;
    size_t bytes = 0;
};

static LoglikWs loglik_ws_layout(void *base, int64_t n, int precision, int want_grad) {
    LoglikWs w;
    const int64_t np = padded(n);
    Carve c(base);
    w.A = c.take<double>((size_t)np * (size_t)np);
    w.r = c.take<double>((size_t)np);
    w.v = c.take<double>((size_t)np);
    w.acc = c.take<double>((size_t)np);
    w.s = c.take<double>((size_t)np);
    w.stats = c.take<double>(4);
    w.conv = c.take<int>(4);
    w.tsync = c.take<int>(trsv_sync_ints(np));
    if (want_grad && precision != GP_FP64) w.winv = c.take<double>(chol_winv_doubles(np));
    size_t cb = chol_ws_bytes(np, precision);
    if (want_grad) {  // the inverse and contraction reuse the factorisation's scratch
        size_t gb = grad_ws_bytes(np, precision, slices_of(precision));
        cb = cb > gb ? cb : gb;
    }
    w.chol = c.take<char>(cb);
    w.bytes = (c.off + 255) & ~size_t(255);
    return w;
}

static int run_chol(double *A, int64_t np, int64_t ld, int precision, void *ws, double *winv,
                    int64_t *info, cudaStream_t s, bool lookahead = true) {
    if (precision == GP_FP64) {
        const int ev = prof_start(s);
        GP_TRY(chol_fp64_tiled(A, ld, np, 0, info, s));
        prof_stop(ev, s, GP_PROF_DIAG, (double)np * np * np / 3.0, 0.0);
        return GP_OK;
    }
    if (precision == GP_MIXED_F16 || precision == GP_EMU_FP64)
        return chol_mixed(A, ld, np, slices_of(precision), ws, winv, info, s, lookahead);
    return GP_ERR_INVALID;
}

// fill -> Cholesky -> solves -> reductions; leaves alpha in w.v.
static int loglik_core(const double *d_x, const double *d_y, const double *d_mu, int64_t n,
                       const KernParams &kp, int precision, const LoglikWs &w, double *d_out,
                       int64_t *d_info, cudaStream_t s, bool lookahead = true) {
    const int64_t np = padded(n);
    if (cudaMemsetAsync(d_info, 0, sizeof(int64_t), s) != cudaSuccess) return GP_ERR_CUDA;
    GP_TRY(launch_cov_fill(d_x, n, np, kp, w.A, np, d_info, s));
    GP_TRY(run_chol(w.A, np, np, precision, w.chol, w.winv, d_info, s, lookahead));
    GP_TRY(launch_residual(d_y, d_mu, n, np, w.r, d_info, s));
    if (cudaMemcpyAsync(w.v, w.r, sizeof(double) * np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GP_ERR_CUDA;
    GP_TRY(trsv_persist(w.A, np, n, 0, w.v, w.tsync, d_info, nullptr, s));
    if (precision == GP_FP64) {
        // q = v^T v with v = L^{-1} r (Sec. 2.2.2); then alpha = L^{-T} v
        GP_TRY(launch_loglik_reduce(w.A, np, n, w.v, w.v, nullptr, d_out, d_info, s));
        GP_TRY(trsv_persist(w.A, np, n, 1, w.v, w.tsync, d_info, nullptr, s));
        return GP_OK;
    }
    // mixed: alpha from the low-precision factor, refined against the FP64
    // matrix-free residual; q = r^T alpha with the refined alpha
    GP_TRY(trsv_persist(w.A, np, n, 1, w.v, w.tsync, d_info, nullptr, s));
    GP_TRY(refine_alpha(d_x, n, np, kp, w.A, np, w.r, w.v, w.acc, w.s, w.stats, w.conv, w.tsync,
                        REFINE_EVALS, REFINE_TOL, d_info, s));
    GP_TRY(launch_loglik_reduce(w.A, np, n, w.r, w.v, w.stats, d_out, d_info, s));
    return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" {

int gp_abi_version(void) { return GP_ABI_VERSION; }

int64_t gp_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *gp_status_string(int status) {
    switch (status) {
        case GP_OK: return "ok";
        case GP_ERR_NOT_PD: return "matrix not positive definite";
        case GP_ERR_INVALID: return "invalid argument";
        case GP_ERR_CUDA: return "CUDA error";
        case GP_ERR_TIMEOUT: return "device wait timed out";
        case GP_ERR_WORKSPACE: return "workspace missing or too small";
        case GP_ERR_TOO_LARGE: return "n exceeds the static scratch of gp_loglik_noalloc";
        default: return "unknown status";
    }
}

int64_t gp_padded_order(int64_t n) { return padded(n); }

size_t gp_chol_workspace_bytes(int64_t n, int precision) {
    if (n < 1 || !precision_ok(precision)) return 0;
    return chol_ws_bytes(padded(n), precision);
}

size_t gp_workspace_bytes(int64_t n, int precision, int want_grad) {
    if (n < 1 || !precision_ok(precision)) return 0;
    return loglik_ws_layout(nullptr, n, precision, want_grad).bytes;
}

int gp_cov_fill(const double *d_x, int64_t n, const gp_params *prm, int precision, double *d_C,
                int64_t ldc, void *stream) {
    if (n < 1 || !d_x || !d_C || !params_ok(prm) || !precision_ok(precision) || ldc < padded(n))
        return GP_ERR_INVALID;
    KernParams kp = make_kern(*prm, precision != GP_FP64);
    return launch_cov_fill(d_x, n, padded(n), kp, d_C, ldc, nullptr, (cudaStream_t)stream);
}

int gp_chol(double *d_C, int64_t n, int64_t ldc, int precision, void *d_ws, size_t ws_bytes,
            int64_t *d_info, void *stream) {
    if (n < 1 || !d_C || !d_info || ldc < padded(n) || !precision_ok(precision))
        return GP_ERR_INVALID;
    size_t need = gp_chol_workspace_bytes(n, precision);
    if (need > 0 && (!d_ws || ws_bytes < need)) return GP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_info, 0, sizeof(int64_t), s) != cudaSuccess) return GP_ERR_CUDA;
    return run_chol(d_C, padded(n), ldc, precision, d_ws, nullptr, d_info, s);
}

int gp_backsolve(const double *d_L, int64_t n, int64_t ldc, int trans, const double *d_b,
                 double *d_out, void *stream) {
    if (n < 1 || !d_L || !d_b || !d_out || ldc < padded(n) || (trans != 0 && trans != 1))
        return GP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_out != d_b &&
        cudaMemcpyAsync(d_out, d_b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GP_ERR_CUDA;
    return trsv_blocked(d_L, ldc, n, trans, d_out, nullptr, s);
}

int gp_mult_chol(const double *d_L, int64_t n, int64_t ldc, const double *d_z, double *d_out,
                 void *stream) {
    if (n < 1 || !d_L || !d_z || !d_out || d_z == d_out || ldc < padded(n)) return GP_ERR_INVALID;
    return lower_matvec(d_L, ldc, n, d_z, d_out, (cudaStream_t)stream);
}

int gp_loglik(const double *d_x, const double *d_y, const double *d_mu, int64_t n,
              const gp_params *prm, int precision, void *d_ws, size_t ws_bytes, double *d_out,
              double *d_alpha, int64_t *d_info, void *stream) {
    if (n < 1 || !d_x || !d_y || !d_out || !d_info || !params_ok(prm) || !precision_ok(precision))
        return GP_ERR_INVALID;
    LoglikWs w = loglik_ws_layout(d_ws, n, precision, 0);
    if (!d_ws || ws_bytes < w.bytes) return GP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    KernParams kp = make_kern(*prm, precision != GP_FP64);
    GP_TRY(loglik_core(d_x, d_y, d_mu, n, kp, precision, w, d_out, d_info, s));
    if (d_alpha &&
        cudaMemcpyAsync(d_alpha, w.v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GP_ERR_CUDA;
    return GP_OK;
}

int gp_loglik_grad(const double *d_x, const double *d_y, const double *d_mu, int64_t n,
                   const gp_params *prm, int precision, void *d_ws, size_t ws_bytes, double *d_out,
                   double *d_alpha, double *d_grad, int64_t *d_info, void *stream) {
    if (n < 1 || !d_x || !d_y || !d_out || !d_grad || !d_info || !params_ok(prm) ||
        !precision_ok(precision))
        return GP_ERR_INVALID;
    LoglikWs w = loglik_ws_layout(d_ws, n, precision, 1);
    if (!d_ws || ws_bytes < w.bytes) return GP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = padded(n);
    KernParams kp = make_kern(*prm, precision != GP_FP64);
    GP_TRY(loglik_core(d_x, d_y, d_mu, n, kp, precision, w, d_out, d_info, s));
    GP_TRY(chol_inverse(w.A, np, np, precision, slices_of(precision), w.chol, w.winv, d_info, s));
    GP_TRY(grad_contract(d_x, n, np, kp, w.A, np, w.v, w.chol, precision, slices_of(precision), d_grad,
                         d_info, s));
    if (d_alpha &&
        cudaMemcpyAsync(d_alpha, w.v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GP_ERR_CUDA;
    return GP_OK;
}

// ---------------------------------------------------------------------------
// The paper's example model (product Matern nu = 2, per-phase random effect,
// known per-point variances): the common path with the product model's fill,
// refinement product and gradient (product.cu).
// ---------------------------------------------------------------------------
static bool product_params_ok(const gp_product_params *p) {
    if (!p) return false;
    if (!(p->sigma2 > 0.0) || !(p->rho_t > 0.0) || !(p->rho_w > 0.0) || !(p->tau2 >= 0.0))
        return false;
    return isfinite(p->sigma2) && isfinite(p->rho_t) && isfinite(p->rho_w) && isfinite(p->tau2);
}

int gp_loglik_product(const double *d_x, const double *d_y, const double *d_mu, const double *d_v,
                      int64_t n, const gp_product_params *prm, int precision, void *d_ws,
                      size_t ws_bytes, double *d_out, double *d_alpha, double *d_grad,
                      int64_t *d_info, void *stream) {
    if (n < 1 || !d_x || !d_y || !d_out || !d_info || !product_params_ok(prm) ||
        !precision_ok(precision))
        return GP_ERR_INVALID;
    const int want_grad = d_grad ? 1 : 0;
    LoglikWs w = loglik_ws_layout(d_ws, n, precision, want_grad);
    if (!d_ws || ws_bytes < w.bytes) return GP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = padded(n);
    gp_params base{GP_KERNEL_EXP, prm->sigma2, 1.0, prm->tau2};
    KernParams kp = make_kern(base, false);
    kp.product = 1;
    kp.prod_st = 2.0 / prm->rho_t;  // Matern nu = 2: a = sqrt(2 nu) d / rho
    kp.prod_sw = 2.0 / prm->rho_w;
    kp.prod_v = d_v;
    kp.diag = prm->sigma2 + prm->tau2;
    GP_TRY(loglik_core(d_x, d_y, d_mu, n, kp, precision, w, d_out, d_info, s));
    if (want_grad) {
        GP_TRY(chol_inverse(w.A, np, np, precision, slices_of(precision), w.chol, w.winv, d_info, s));
        GP_TRY(grad_contract(d_x, n, np, kp, w.A, np, w.v, w.chol, precision, slices_of(precision),
                             d_grad, d_info, s));
    }
    if (d_alpha &&
        cudaMemcpyAsync(d_alpha, w.v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GP_ERR_CUDA;
    return GP_OK;
}

// ---------------------------------------------------------------------------
// Batched evaluation: independent problems on a pool of library streams,
// forked from and joined back to the caller's stream with events, so that a
// capture of the caller's stream records the whole batch as one graph.
// ---------------------------------------------------------------------------
size_t gp_batched_workspace_bytes(int nprob, const int64_t *h_n, int precision) {
    if (nprob < 1 || !h_n || !precision_ok(precision)) return 0;
    for (int i = 0; i < nprob; ++i)
        if (h_n[i] < 1) return 0;
    if (precision != GP_EMU_FP64) return dag_workspace_bytes(nprob, h_n, precision == GP_MIXED_F16);
    size_t tot = 0;
    for (int i = 0; i < nprob; ++i) {
        tot += (loglik_ws_layout(nullptr, h_n[i], precision, 1).bytes + 255) & ~size_t(255);
    }
    return tot;
}

}  // extern "C"

namespace gp {

constexpr int BATCH_STREAMS = 24;

struct StreamPool {
    cudaStream_t s[BATCH_STREAMS];
    cudaEvent_t done[BATCH_STREAMS];
    cudaEvent_t fork;
};

// One pool per device, created on first use and kept for the process.
static int batch_pool(StreamPool **out) {
    static std::mutex mu;
    static StreamPool *pools[64] = {};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        StreamPool *p = new StreamPool();
        if (cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess) {
            delete p;
            return GP_ERR_CUDA;
        }
        for (int k = 0; k < BATCH_STREAMS; ++k) {
            if (cudaStreamCreateWithFlags(&p->s[k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->done[k], cudaEventDisableTiming) != cudaSuccess) {
                delete p;
                return GP_ERR_CUDA;
            }
        }
        pools[dev] = p;
    }
    *out = pools[dev];
    return GP_OK;
}

}  // namespace gp

extern "C" {

int gp_loglik_grad_batched(int nprob, const int64_t *h_n, const double *const *h_dx,
                           const double *const *h_dy, const double *const *h_dmu,
                           const gp_params *h_prm, int precision, void *d_ws, size_t ws_bytes,
                           double *d_out, double *d_grad, int64_t *d_info, void *stream) {
    if (nprob < 1 || !h_n || !h_dx || !h_dy || !h_prm || !d_out || !d_grad || !d_info ||
        !precision_ok(precision))
        return GP_ERR_INVALID;
    for (int i = 0; i < nprob; ++i)
        if (h_n[i] < 1 || !h_dx[i] || !h_dy[i] || !params_ok(&h_prm[i])) return GP_ERR_INVALID;
    const size_t need = gp_batched_workspace_bytes(nprob, h_n, precision);
    if (!d_ws || ws_bytes < need) return GP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision != GP_EMU_FP64) {
        // one persistent task-graph launch (FP64 CUDA-core tiles, or tcgen05 slice tiles)
        std::vector<KernParams> kps(nprob);
        for (int i = 0; i < nprob; ++i) kps[i] = make_kern(h_prm[i], precision != GP_FP64);
        const int mixed = precision == GP_MIXED_F16;
        return dag_run(nprob, h_n, h_dx, h_dy, h_dmu, kps.data(), mixed, mixed ? dag_fp64_max_n() : 0,
                       d_ws, ws_bytes, d_out, d_grad, d_info, s);
    }
    StreamPool *pool = nullptr;
    GP_TRY(batch_pool(&pool));
    // workspace offsets in problem order
    std::vector<size_t> off(nprob);
    size_t acc = 0;
    for (int i = 0; i < nprob; ++i) {
        off[i] = acc;
        acc += (loglik_ws_layout(nullptr, h_n[i], precision, 1).bytes + 255) & ~size_t(255);
    }
    // longest-processing-time assignment of problems (cost ~ n^3) to streams
    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return h_n[a] > h_n[b]; });
    const int ns = nprob < BATCH_STREAMS ? nprob : BATCH_STREAMS;
    std::vector<double> load(ns, 0.0);
    std::vector<std::vector<int>> lists(ns);
    for (int i : order) {
        int best = 0;
        for (int k = 1; k < ns; ++k)
            if (load[k] < load[best]) best = k;
        load[best] += (double)h_n[i] * h_n[i] * h_n[i];
        lists[best].push_back(i);
    }
    if (cudaEventRecord(pool->fork, s) != cudaSuccess) return GP_ERR_CUDA;
    int status = GP_OK;
    for (int k = 0; k < ns; ++k) {
        cudaStream_t sk = pool->s[k];
        if (cudaStreamWaitEvent(sk, pool->fork, 0) != cudaSuccess) return GP_ERR_CUDA;
        for (int i : lists[k]) {
            const int64_t n = h_n[i];
            const int64_t np = padded(n);
            LoglikWs w = loglik_ws_layout(static_cast<char *>(d_ws) + off[i], n, precision, 1);
            KernParams kp = make_kern(h_prm[i], precision != GP_FP64);
            const double *mu = h_dmu ? h_dmu[i] : nullptr;
            // many problems run side by side here: no lookahead side stream
            int st = loglik_core(h_dx[i], h_dy[i], mu, n, kp, precision, w, d_out + 4 * i,
                                 d_info + i, sk, false);
            if (st == GP_OK)
                st = chol_inverse(w.A, np, np, precision, slices_of(precision), w.chol, w.winv,
                                  d_info + i, sk);
            if (st == GP_OK)
                st = grad_contract(h_dx[i], n, np, kp, w.A, np, w.v, w.chol, precision,
                                   slices_of(precision), d_grad + 3 * i, d_info + i, sk);
            if (st != GP_OK && status == GP_OK) status = st;
        }
        // join even after a launch error, so that the caller's stream stays ordered
        if (cudaEventRecord(pool->done[k], sk) != cudaSuccess ||
            cudaStreamWaitEvent(s, pool->done[k], 0) != cudaSuccess)
            return GP_ERR_CUDA;
    }
    return status;
}

void gp_batched_profile(int on) { dag_set_profile(on); }

int gp_batched_set_wait_limit(double seconds) {
    if (!(seconds >= 1e-3 && seconds <= 600.0)) return GP_ERR_INVALID;
    return dag_set_wait_ns((uint64_t)(seconds * 1e9));
}

int gp_batched_test_unset_tile(int problem, int64_t tile_row, int64_t tile_col) {
    return dag_set_unset_tile(problem, tile_row, tile_col);
}

int gp_batched_set_tile_policy(int64_t fp64_max_n) {
    if (fp64_max_n < 0) return GP_ERR_INVALID;
    dag_set_fp64_max_n(fp64_max_n);
    return GP_OK;
}

int64_t gp_batched_tile_policy(void) { return dag_fp64_max_n(); }

int gp_batched_plan_check(int nprob, const int64_t *h_n, int precision, int64_t fp64_max_n,
                          int64_t *h_ntasks, int64_t *h_bad_order, int64_t *h_bad_slots) {
    if (!h_n || !(precision == GP_FP64 || precision == GP_MIXED_F16) || fp64_max_n < 0)
        return GP_ERR_INVALID;
    return dag_plan_check(nprob, h_n, precision == GP_MIXED_F16, fp64_max_n, h_ntasks, h_bad_order,
                          h_bad_slots);
}

// The tile autotuner of the mixed batched launch: time the caller's batch
// with every candidate threshold (problems with n <= threshold on FP64
// 64 x 64 tiles, the others on tensor-core 128 x 128 tiles), one warm-up
// and two timed launches each, keep the fastest as this device's policy.
int gp_batched_autotune(int nprob, const int64_t *h_n, const double *const *h_dx,
                        const double *const *h_dy, const double *const *h_dmu,
                        const gp_params *h_prm, int precision, void *d_ws, size_t ws_bytes,
                        double *d_out, double *d_grad, int64_t *d_info, void *stream,
                        int64_t *h_choice, double *h_ms, int *h_ncand) {
    if (nprob < 1 || !h_n || !h_dx || !h_dy || !h_prm || !d_out || !d_grad || !d_info ||
        !h_choice || precision != GP_MIXED_F16)
        return GP_ERR_INVALID;
    for (int i = 0; i < nprob; ++i)
        if (h_n[i] < 1 || !h_dx[i] || !h_dy[i] || !params_ok(&h_prm[i])) return GP_ERR_INVALID;
    if (!d_ws || ws_bytes < gp_batched_workspace_bytes(nprob, h_n, precision)) return GP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<KernParams> kps(nprob);
    for (int i = 0; i < nprob; ++i) kps[i] = make_kern(h_prm[i], true);
    int64_t nmax = 0;
    for (int i = 0; i < nprob; ++i) nmax = std::max(nmax, h_n[i]);
    std::vector<int64_t> cand{0};
    for (int64_t t : {256, 384, 512, 768, 1024, 1536})
        if (t < nmax) cand.push_back(t);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GP_ERR_CUDA;
    int status = GP_OK;
    double best_ms = 1e300;
    int64_t best = 0;
    for (size_t q = 0; q < cand.size() && status == GP_OK; ++q) {
        double ms_min = 1e300;
        for (int rep = 0; rep < 3 && status == GP_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) status = GP_ERR_CUDA;
            if (status == GP_OK)
                status = dag_run(nprob, h_n, h_dx, h_dy, h_dmu, kps.data(), 1, cand[q], d_ws, ws_bytes,
                                 d_out, d_grad, d_info, s);
            if (status == GP_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                    cudaEventSynchronize(e1) != cudaSuccess))
                status = GP_ERR_CUDA;
            float ms = 0.0f;
            if (status == GP_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) status = GP_ERR_CUDA;
            if (rep > 0) ms_min = std::min(ms_min, (double)ms);  // the first run warms up
        }
        if (h_ms && q < 8) h_ms[q] = ms_min;
        if (ms_min < best_ms) {
            best_ms = ms_min;
            best = cand[q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != GP_OK) return status;
    if (h_ncand) *h_ncand = (int)std::min<size_t>(cand.size(), 8);
    dag_set_fp64_max_n(best);
    *h_choice = best;
    return GP_OK;
}

int gp_batched_task_stats(const void *d_ws, unsigned long long *h_out) {
    if (!d_ws || !h_out) return GP_ERR_INVALID;
    return dag_stats(d_ws, h_out);
}

size_t gp_predict_workspace_bytes(int64_t n, int64_t m, int want_var) {
    if (n < 1 || m < 1) return 0;
    return predict_ws_bytes(n, m, want_var);
}

int gp_predict(const double *d_x, int64_t n, const double *d_xnew, int64_t m, const gp_params *prm,
               const double *d_alpha, const double *d_L, int64_t ldl, double mu_new, double *d_mean,
               double *d_var, void *d_ws, size_t ws_bytes, int64_t *d_info, void *stream) {
    if (n < 1 || m < 1 || !d_x || !d_xnew || !d_alpha || !d_mean || !d_info || !params_ok(prm) ||
        !isfinite(mu_new))
        return GP_ERR_INVALID;
    if (d_var) {
        if (!d_L || ldl < padded(n)) return GP_ERR_INVALID;
        if (!d_ws || ws_bytes < predict_ws_bytes(n, m, 1)) return GP_ERR_WORKSPACE;
    }
    KernParams kp = make_kern(*prm);
    return predict_run(d_x, n, d_xnew, m, kp, d_alpha, d_L, ldl, mu_new, d_mean, d_var, d_ws, d_info,
                       (cudaStream_t)stream);
}

int gp_rng_normal(int64_t n, int64_t r, uint64_t seed, uint64_t stream_id, uint64_t first,
                  double *d_out, int64_t ldo, void *stream) {
    if (n < 1 || r < 1 || !d_out || ldo < n) return GP_ERR_INVALID;
    return rng_normals(n, n, r, seed, stream_id, first, d_out, ldo, (cudaStream_t)stream);
}

size_t gp_simulate_workspace_bytes(int64_t n, int64_t r) {
    if (n < 1 || r < 1) return 0;
    return simulate_ws_bytes(n, r);
}

int gp_simulate(const double *d_L, int64_t n, int64_t ldl, int64_t r, uint64_t seed, uint64_t first,
                double mu, double *d_out, int64_t ldo, void *d_ws, size_t ws_bytes, void *stream) {
    if (n < 1 || r < 1 || !d_L || !d_out || ldl < n || ldo < n || !isfinite(mu))
        return GP_ERR_INVALID;
    if (!d_ws || ws_bytes < simulate_ws_bytes(n, r)) return GP_ERR_WORKSPACE;
    return simulate_run(d_L, n, ldl, r, seed, first, mu, d_out, ldo, d_ws, (cudaStream_t)stream);
}

size_t gp_simulate_conditional_workspace_bytes(int64_t n, int64_t m, int64_t r) {
    if (n < 1 || m < 1 || r < 1) return 0;
    return simulate_cond_ws_bytes(n, m, r);
}

int gp_simulate_conditional(const double *d_x, int64_t n, const double *d_xnew, int64_t m,
                            const gp_params *prm, const double *d_alpha, const double *d_L,
                            int64_t ldl, double mu_new, int64_t r, uint64_t seed, uint64_t first,
                            double *d_out, int64_t ldo, void *d_ws, size_t ws_bytes,
                            int64_t *d_info, void *stream) {
    if (n < 1 || m < 1 || r < 1 || !d_x || !d_xnew || !d_alpha || !d_L || !d_out || !d_info ||
        !params_ok(prm) || ldl < padded(n) || ldo < m || !isfinite(mu_new))
        return GP_ERR_INVALID;
    if (!d_ws || ws_bytes < simulate_cond_ws_bytes(n, m, r)) return GP_ERR_WORKSPACE;
    return simulate_cond_run(d_x, n, d_xnew, m, *prm, d_alpha, d_L, ldl, mu_new, r, seed, first,
                             d_out, ldo, d_ws, d_info, (cudaStream_t)stream);
}

size_t gp_syrk_workspace_bytes(int64_t m, int64_t k, int precision) {
    if (m < 1 || k < 1 || !precision_ok(precision)) return 0;
    return syrk_ws_bytes(m, k, precision, slices_of(precision));
}

int gp_syrk_lower(double *d_C, int64_t ldc, const double *d_P, int64_t ldp, int64_t m, int64_t k,
                  int precision, void *d_ws, size_t ws_bytes, int64_t *d_info, void *stream) {
    if (m < 1 || k < 1 || !d_C || !d_P || ldc < m || ldp < m || !precision_ok(precision))
        return GP_ERR_INVALID;
    size_t need = syrk_ws_bytes(m, k, precision, slices_of(precision));
    if (need > 0 && (!d_ws || ws_bytes < need)) return GP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_info && cudaMemsetAsync(d_info, 0, sizeof(int64_t), s) != cudaSuccess) return GP_ERR_CUDA;
    return syrk_lower(d_C, ldc, d_P, ldp, m, k, precision, slices_of(precision), d_ws, d_info, s);
}

}  // extern "C"
