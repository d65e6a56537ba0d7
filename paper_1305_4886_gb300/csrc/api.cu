// api.cu -- the extern "C" entry points of libgp (declared in include/gp.h):
// argument checks, workspace carving and the launch sequence of each step.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "kern.cuh"

namespace gp {

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

static bool precision_ok(int p) { return p == GP_FP64 || p == GP_MIXED_BF16; }

int64_t padded(int64_t n) { return n < 1 ? 0 : round_up(n, PAD); }

// Workspace of the factorisation (beyond the matrix itself).
struct CholWs {
    size_t bytes = 0;
};

static size_t chol_ws_layout(int64_t np, int precision, Carve &c) {
    (void)np;
    (void)precision;
    (void)c;
    return c.off;
}

struct LoglikWs {
    double *A = nullptr;
    double *r = nullptr;
    void *chol = nullptr;
    size_t bytes = 0;
};

static LoglikWs loglik_ws_layout(void *base, int64_t n, int precision, int want_grad) {
    (void)want_grad;
    LoglikWs w;
    const int64_t np = padded(n);
    Carve c(base);
    w.A = c.take<double>((size_t)np * (size_t)np);
    w.r = c.take<double>((size_t)np);
    Carve cc(nullptr);
    size_t chol_bytes = chol_ws_layout(np, precision, cc);
    w.chol = c.take<char>(chol_bytes);
    w.bytes = c.off;
    return w;
}

static int run_chol(double *A, int64_t np, int64_t ld, int precision, void *ws, int64_t *info,
                    cudaStream_t s) {
    (void)ws;
    if (precision == GP_FP64) return chol_fp64_tiled(A, ld, np, 0, info, s);
    return GP_ERR_INVALID;
}

}  // namespace gp

using namespace gp;

extern "C" {

int gp_abi_version(void) { return GP_ABI_VERSION; }

const char *gp_status_string(int status) {
    switch (status) {
        case GP_OK: return "ok";
        case GP_ERR_NOT_PD: return "matrix not positive definite";
        case GP_ERR_INVALID: return "invalid argument";
        case GP_ERR_CUDA: return "CUDA error";
        case GP_ERR_TIMEOUT: return "device wait timed out";
        case GP_ERR_WORKSPACE: return "workspace missing or too small";
        default: return "unknown status";
    }
}

int64_t gp_padded_order(int64_t n) { return padded(n); }

size_t gp_chol_workspace_bytes(int64_t n, int precision) {
    if (n < 1 || !precision_ok(precision)) return 0;
    Carve c(nullptr);
    return chol_ws_layout(padded(n), precision, c);
}

size_t gp_workspace_bytes(int64_t n, int precision, int want_grad) {
    if (n < 1 || !precision_ok(precision)) return 0;
    return loglik_ws_layout(nullptr, n, precision, want_grad).bytes;
}

int gp_cov_fill(const double *d_x, int64_t n, const gp_params *prm, double *d_C, int64_t ldc,
                void *stream) {
    if (n < 1 || !d_x || !d_C || !params_ok(prm) || ldc < padded(n)) return GP_ERR_INVALID;
    KernParams kp = make_kern(*prm);
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
    return run_chol(d_C, padded(n), ldc, precision, d_ws, d_info, s);
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
    const int64_t np = padded(n);
    KernParams kp = make_kern(*prm);
    if (cudaMemsetAsync(d_info, 0, sizeof(int64_t), s) != cudaSuccess) return GP_ERR_CUDA;
    GP_TRY(launch_cov_fill(d_x, n, np, kp, w.A, np, d_info, s));
    GP_TRY(run_chol(w.A, np, np, precision, w.chol, d_info, s));
    GP_TRY(launch_residual(d_y, d_mu, n, np, w.r, d_info, s));
    GP_TRY(trsv_blocked(w.A, np, n, 0, w.r, d_info, s));
    GP_TRY(launch_loglik_reduce(w.A, np, n, w.r, d_out, d_info, s));
    if (d_alpha) {
        if (cudaMemcpyAsync(d_alpha, w.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return GP_ERR_CUDA;
        GP_TRY(trsv_blocked(w.A, np, n, 1, d_alpha, d_info, s));
    }
    return GP_OK;
}

}  // extern "C"
