// noalloc.cu -- gp_loglik_noalloc: the FP64 log-likelihood for small n with
// its scratch in a static device array instead of a caller-provided
// workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// log-likelihood: code running while a stream is being captured into a CUDA
// graph (an allocation there breaks the capture), real-time or embedded
// callers whose device memory budget is fixed when they start, and plug-ins
// inside a host application that owns every device allocation.  This entry
// point needs no workspace and calls no allocating routine.
//
// The scratch lives in one file-scope array of GP_NOALLOC_SCRATCH_BYTES
// (about 2.1 MB), enough for n <= GP_NOALLOC_MAX_N = 512.  Every GPU that
// loads this library holds it until the process exits.  Host code cannot use
// the array's name as a device address, so the first call on each device
// looks up the device address with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before any stream capture
// begins.  All calls on a device share the array: two calls whose work
// overlaps on the GPU (different streams, or different host threads) race
// and corrupt each other's results, so serialise them.  Each call rewrites
// every scratch entry it reads before reading it, so nothing left over from
// an earlier call affects the result.
#include <mutex>

#include "internal.h"
#include "kern.cuh"

namespace gp {

constexpr int64_t NA_N = GP_NOALLOC_MAX_N;
constexpr size_t NA_MAT = (size_t)NA_N * NA_N;  // the n_p x n_p matrix (n_p <= NA_N)
constexpr size_t NA_VEC = (size_t)NA_N;          // r and v
constexpr size_t NA_DOUBLES = NA_MAT + 2 * NA_VEC + 64;  // + room for the solve flags
static_assert(NA_DOUBLES * sizeof(double) == GP_NOALLOC_SCRATCH_BYTES,
              "GP_NOALLOC_SCRATCH_BYTES must match the scratch layout");

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

namespace {
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
void *g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return GP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GP_ERR_CUDA;
        g_na_ptr[dev] = p;
    }
    *out = static_cast<double *>(g_na_ptr[dev]);
    return GP_OK;
}

bool na_params_ok(const gp_params *p) {
    if (!p) return false;
    if (p->kernel < GP_KERNEL_EXP || p->kernel > GP_KERNEL_MATERN52) return false;
    if (!(p->sigma2 > 0.0) || !(p->rho > 0.0) || !(p->tau2 >= 0.0)) return false;
    return isfinite(p->sigma2) && isfinite(p->rho) && isfinite(p->tau2);
}
}  // namespace

}  // namespace gp

using namespace gp;

extern "C" int gp_loglik_noalloc(const double *d_x, const double *d_y, const double *d_mu,
                                 int64_t n, const gp_params *prm, double *d_out, double *d_alpha,
                                 int64_t *d_info, void *stream) {
    if (n < 1 || !d_x || !d_y || !d_out || !d_info || !na_params_ok(prm)) return GP_ERR_INVALID;
    if (n > NA_N) return GP_ERR_TOO_LARGE;
    double *base = nullptr;
    GP_TRY(noalloc_scratch(&base));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = round_up(n, PAD);
    double *A = base;  // ld = np
    double *r = base + NA_MAT;
    double *v = r + NA_VEC;
    int *tsync = reinterpret_cast<int *>(v + NA_VEC);
    KernParams kp = make_kern(*prm);
    if (cudaMemsetAsync(d_info, 0, sizeof(int64_t), s) != cudaSuccess) return GP_ERR_CUDA;
    GP_TRY(launch_cov_fill(d_x, n, np, kp, A, np, d_info, s));
    GP_TRY(chol_fp64_tiled(A, np, np, 0, d_info, s));
    GP_TRY(launch_residual(d_y, d_mu, n, np, r, d_info, s));
    if (cudaMemcpyAsync(v, r, sizeof(double) * np, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GP_ERR_CUDA;
    GP_TRY(trsv_persist(A, np, n, 0, v, tsync, d_info, nullptr, s));
    GP_TRY(launch_loglik_reduce(A, np, n, v, v, nullptr, d_out, d_info, s));
    GP_TRY(trsv_persist(A, np, n, 1, v, tsync, d_info, nullptr, s));
    if (d_alpha &&
        cudaMemcpyAsync(d_alpha, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return GP_ERR_CUDA;
    return GP_OK;
}
