/*
 * gp.h -- C ABI of libgp, a GB300 (sm_103a) library for the Gaussian-process
 * marginal log-likelihood of Paciorek et al., "Parallelizing Gaussian Process
 * Calculations in R" (arXiv:1305.4886).
 *
 * The operation (Sec. 1): for locations x_1..x_n, data y and mean mu,
 *     C(theta) = C_g(theta) + C_y(theta)            (covariance + nugget)
 *     L L^T    = C(theta)                           (Cholesky, no pivoting)
 *     v        = L^{-1} (y - mu)                    (forward solve)
 *     logdet   = 2 sum_i log L_ii,  q = v^T v        (Sec. 2.2.2)
 *     loglik   = -logdet/2 - q/2 - (n/2) log(2 pi)
 *
 * Conventions shared by every entry point
 *   - Pointers prefixed d_ are device pointers; h_ are host pointers.  The
 *     caller owns every buffer, including workspaces; the library never
 *     allocates device memory in these calls and keeps no hidden state
 *     between them.  The tensor-core factorisations (GP_MIXED_F16,
 *     GP_EMU_FP64 in gp_chol, gp_loglik, gp_loglik_grad) run their
 *     diagonal blocks on a library side stream, forked from and joined back
 *     to the caller's stream with events: that stream and its two events
 *     are created on the first such call on a device (make it outside a
 *     stream capture) and kept for the process.
 *   - Matrices are FP64, column-major, lower triangle referenced, leading
 *     dimension ld >= gp_padded_order(n).  The padded order n_p rounds n up
 *     to a multiple of GP_PAD (the block padding of Sec. 2.2); rows/columns
 *     n..n_p-1 are owned by the library and hold the identity, so they add
 *     log 1 = 0 to logdet and 0 to q.  Entries above the diagonal are never
 *     read and may be overwritten inside diagonal tiles.
 *   - Locations are n points x 2 coordinates, interleaved (x_i1, x_i2).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     is asynchronous on it: the host return code reports argument checks
 *     and launch errors only.  Failures found on the device go to the
 *     caller's int64 *d_info, which the caller reads after its own sync:
 *        0      success
 *        k + 1  the unpivoted Cholesky met a pivot <= 0 (or NaN) at global
 *               column k -- the failure mode of Sec. 5
 *        -1     a bounded device-side wait gave up (timeout)
 *        -2     non-finite input (location, data or mean)
 *     When *d_info != 0 the scalar outputs are NaN.
 *   - Kernel parameters are on the natural scale: sigma2 > 0, rho > 0,
 *     tau2 >= 0, all finite.  Gradients are with respect to
 *     theta = (log sigma2, log rho, log tau2).
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GP_ABI_VERSION 2
#define GP_PAD 128 /* padding granularity of n (rows/columns of one tile) */

typedef enum {
    GP_OK = 0,
    GP_ERR_NOT_PD = 1,    /* reserved: device-side detection goes to d_info */
    GP_ERR_INVALID = 2,   /* bad argument (sizes, parameters, NULL pointers) */
    GP_ERR_CUDA = 3,      /* a CUDA launch or runtime call failed */
    GP_ERR_TIMEOUT = 4,   /* reserved: device-side detection goes to d_info */
    GP_ERR_WORKSPACE = 5, /* workspace missing or smaller than required */
    GP_ERR_TOO_LARGE = 6  /* n above GP_NOALLOC_MAX_N for gp_loglik_noalloc */
} gp_status;

/* Covariance functions k(u), u = d / rho, d Euclidean distance (Sec. 1;
 * Matern in the Rasmussen & Williams parameterisation):
 *   EXP       exp(-u)
 *   MATERN32  (1 + a) exp(-a),           a = sqrt(3) u
 *   MATERN52  (1 + a + a^2/3) exp(-a),   a = sqrt(5) u                     */
typedef enum { GP_KERNEL_EXP = 0, GP_KERNEL_MATERN32 = 1, GP_KERNEL_MATERN52 = 2 } gp_kernel;

/* Arithmetic of the factorisation.
 *   GP_FP64        every step in FP64 on the CUDA cores.
 *   GP_MIXED_F16  the mixed form: FP64 diagonal blocks (their 64 x 64
 *                  diagonal tiles factored in double-float, about 48 bits,
 *                  the precision of the pending updates), pivots,
 *                  log-determinant and residuals; the off-diagonal panel
 *                  solve, the trailing SYRK updates and the gradient's
 *                  inverse run on the tcgen05 tensor cores over three
 *                  16-bit slices of each FP64 operand row (an integer
 *                  leading slice on the row's grid plus two FP16
 *                  remainders, about 32 bits; 6 slice products, FP32
 *                  accumulation with the leading products exact), pending
 *                  trailing updates kept as FP32 pairs (double-float),
 *                  followed by iterative refinement of alpha against a
 *                  matrix-free FP64 residual.
 *   GP_EMU_FP64    the same structure with FP64-grade contractions: five
 *                  integer-valued BF16 slices per operand row (40 bits),
 *                  15 slice products, the three leading product groups
 *                  accumulated exactly in their own FP32 accumulators.
 *                  About 2.5x the tensor work of GP_MIXED_F16.            */
typedef enum { GP_FP64 = 0, GP_MIXED_F16 = 1, GP_EMU_FP64 = 2 } gp_precision;

typedef struct {
    int32_t kernel; /* gp_kernel */
    double sigma2;  /* marginal variance of the latent process, > 0 */
    double rho;     /* range, > 0 */
    double tau2;    /* nugget (diagonal of C_y), >= 0 */
} gp_params;

/* ---- queries (pure host functions) ------------------------------------ */

int gp_abi_version(void);
const char *gp_status_string(int status);

/* n rounded up to a multiple of GP_PAD; 0 for n < 1. */
int64_t gp_padded_order(int64_t n);

/* Bytes of device workspace that gp_loglik (want_grad = 0) or
 * gp_loglik_grad (want_grad = 1) needs for this n and precision; 0 for an
 * invalid request.  The first gp_padded_order(n)^2 doubles of the workspace
 * hold the matrix (column-major, ld = n_p): after gp_loglik they hold the
 * Cholesky factor L, after gp_loglik_grad the lower triangle of C^{-1}.   */
size_t gp_workspace_bytes(int64_t n, int precision, int want_grad);

/* Bytes of workspace gp_chol needs for this n and precision. */
size_t gp_chol_workspace_bytes(int64_t n, int precision);

/* ---- the steps of the path ------------------------------------------- */

/* Covariance fill (Sec. 1: C = C_g + C_y; Sec. 2.3.5: entries built from a
 * covariance function at given indices).  Writes the lower tiles of the
 * n_p x n_p matrix d_C (ld = ldc): C_ij = sigma2 k(d_ij/rho) for i != j,
 * C_ii = sigma2 + tau2, identity in the padding.  precision selects the
 * evaluation the factorisations of that precision use: GP_FP64 in FP64;
 * the tensor-core forms in double-float on the FP32 pipe (about 48
 * significant bits: a few hundred FP64 ulps; entries with exp(-d/rho
 * scaled) below 2^-125, all below 1e-33 sigma2, set to 0).                                                               */
int gp_cov_fill(const double *d_x, int64_t n, const gp_params *prm, int precision, double *d_C,
                int64_t ldc, void *stream);

/* Cholesky factorisation L L^T = C in place (Sec. 1; block algorithm of
 * Sec. 2.1): d_C holds the n_p x n_p matrix from gp_cov_fill on entry and
 * L on exit (lower triangle; padding stays identity).  No pivoting: a pivot
 * <= 0 sets *d_info = column + 1 (Sec. 5).  d_ws: gp_chol_workspace_bytes. */
int gp_chol(double *d_C, int64_t n, int64_t ldc, int precision, void *d_ws,
            size_t ws_bytes, int64_t *d_info, void *stream);

/* Triangular solve with the factor (Sec. 1 "backsolve"; the paper's
 * forwardsolve/backsolve pair, Sec. 2.3.2):
 *   trans = 0: d_out = L^{-1} d_b      trans = 1: d_out = L^{-T} d_b.
 * d_b and d_out hold n values; they may alias.                            */
int gp_backsolve(const double *d_L, int64_t n, int64_t ldc, int trans, const double *d_b,
                 double *d_out, void *stream);

/* d_out = L d_z (n values; the paper's multiplication by the Cholesky factor
 * used for simulation, Sec. 2.3.2).  d_z and d_out must not alias.         */
int gp_mult_chol(const double *d_L, int64_t n, int64_t ldc, const double *d_z, double *d_out,
                 void *stream);

/* Log-likelihood (Sec. 1, Sec. 2.2.2).  d_mu: n values or NULL (zero mean).
 * d_out[0..3] = {loglik, logdet, q, refinement residual}; the last is
 * ||r - C alpha||_2 / ||r||_2 after refinement in the tensor-core forms,
 * and 0 in GP_FP64.  d_alpha: n values or NULL; receives C^{-1}(y - mu).  d_ws:
 * gp_workspace_bytes(n, precision, 0); on return its first n_p^2 doubles
 * hold L.                                                                  */
int gp_loglik(const double *d_x, const double *d_y, const double *d_mu, int64_t n,
              const gp_params *prm, int precision, void *d_ws, size_t ws_bytes,
              double *d_out, double *d_alpha, int64_t *d_info, void *stream);

/* Log-likelihood and its gradient (the gradient is not in the paper, whose
 * optimiser uses none).  Same arguments as gp_loglik plus d_grad[3] =
 * d loglik / d(log sigma2, log rho, log tau2), computed as
 *   sum_{i,k} Cbar_ik (dC/dtheta_j)_ik,  Cbar = (alpha alpha^T - C^{-1}) / 2,
 * with C^{-1} formed in place from the factor (blocked TRTRI + LAUUM) and
 * dC/dtheta recomputed tile by tile from the locations.  In the tensor-core
 * forms the inverse's contractions use the tensor cores like the
 * factorisation.
 * d_ws: gp_workspace_bytes(n, precision, 1); on return its first n_p^2
 * doubles hold the lower triangle of C^{-1}.                               */
int gp_loglik_grad(const double *d_x, const double *d_y, const double *d_mu, int64_t n,
                   const gp_params *prm, int precision, void *d_ws, size_t ws_bytes,
                   double *d_out, double *d_alpha, double *d_grad, int64_t *d_info, void *stream);

/* The paper's example model (Sec. 4.2): observation i at phase t_i and log
 * wavelength w_i (the two location coordinates, interleaved as for the other
 * entry points) is a Gaussian-process value plus a random effect of its
 * phase plus measurement error of known variance v_i:
 *   C_ij = sigma2 k(|t_i - t_j| / rho_t) k(|w_i - w_j| / rho_w)
 *          + tau2 [t_i == t_j] + v_i [i == j],
 * k the Matern correlation of smoothness 2 in the Rasmussen & Williams
 * scaling: k(u) = a^2 K_2(a) / 2 with a = 2u (K_2 the modified Bessel
 * function of the second kind; entries with a >= 48, below 1e-18 sigma2,
 * are 0).  "Same phase" is exact equality of the first coordinate.        */
typedef struct {
    double sigma2; /* variance of the latent process, > 0 */
    double rho_t;  /* range in the first coordinate (phase), > 0 */
    double rho_w;  /* range in the second coordinate (log wavelength), > 0 */
    double tau2;   /* variance of the per-phase random effect, >= 0 */
} gp_product_params;

/* Log-likelihood of the product model, and its gradient with respect to
 * (log sigma2, log rho_t, log rho_w, log tau2) when d_grad (4 values) is not
 * NULL.  d_v: n known variances (>= 0), or NULL for none; d_mu, d_out,
 * d_alpha, d_info as gp_loglik.  d_ws: gp_workspace_bytes(n, precision,
 * d_grad != NULL).  Every precision form factors and inverts as for the
 * other models; this model's covariance entries (fill, the refinement's
 * C alpha, the gradient's dC) are evaluated in FP64 in every form, from
 * piecewise Chebyshev tables of a^2 K_2(a) / 2 and a^3 K_1(a) / 2 built once
 * per process on the host (about 1e-15 relative).  Non-finite locations or
 * variances, or a negative variance, set *d_info = -2.                    */
int gp_loglik_product(const double *d_x, const double *d_y, const double *d_mu, const double *d_v,
                      int64_t n, const gp_product_params *prm, int precision, void *d_ws,
                      size_t ws_bytes, double *d_out, double *d_alpha, double *d_grad,
                      int64_t *d_info, void *stream);

/* Batched log-likelihood + gradient of nprob independent problems of uneven
 * n (independent data sets or a theta grid; the paper evaluates one
 * problem per session, Sec. 2.3.4).  Host arrays, one entry per problem:
 * h_n (sizes), h_dx / h_dy (device pointers to locations and data), h_dmu
 * (NULL, or device pointers to means, each NULL = 0), h_prm (parameters).
 * Device outputs: d_out (nprob x 4, as gp_loglik), d_grad (nprob x 3),
 * d_info (nprob, per-problem status as d_info of gp_loglik; -1 also when
 * the launch stopped on a wait limit).  d_ws: gp_batched_workspace_bytes
 * (nprob <= 65535), owned by the caller and not read across calls.
 * GP_FP64 and GP_MIXED_F16 run the whole batch as ONE persistent kernel
 * over a task graph of tile tasks (fill, Cholesky, solves, refinement,
 * inverse, gradient) of every problem, after a few small set-up kernels
 * that copy the problem descriptors (as kernel parameters) and order the
 * tasks; every launch is on `stream`, nothing is allocated and the host
 * never waits, so a capture of `stream` records the batch as one CUDA
 * graph.  GP_EMU_FP64 runs each problem's single-problem launch sequence
 * on a pool of library streams (created on the first such call on a
 * device, forked from and joined back to `stream` with events; make the
 * first call outside a capture).                                          */
size_t gp_batched_workspace_bytes(int nprob, const int64_t *h_n, int precision);
int gp_loglik_grad_batched(int nprob, const int64_t *h_n, const double *const *h_dx,
                           const double *const *h_dy, const double *const *h_dmu,
                           const gp_params *h_prm, int precision, void *d_ws, size_t ws_bytes,
                           double *d_out, double *d_grad, int64_t *d_info, void *stream);

/* Diagnostics of the persistent batched launch.  gp_batched_profile(1)
 * makes later batched calls count SM cycles per task class (off by default,
 * or on with GP_DAG_PROFILE=1 in the environment).  After a synchronisation,
 * gp_batched_task_stats copies the counters of the last batched call on
 * d_ws into h_out[31]: cycles [0..9], of which waiting for inputs [10..19],
 * tasks [20..29] per class (0 off-diagonal Cholesky tile, 1 solve,
 * 2 inverse tile, 3 inverse-product + gradient tile, 4 gradient sum,
 * 5 refinement residual, 6 refinement correction, 7 log-likelihood,
 * 8 diagonal Cholesky tile, 9 refinement residual of a problem already
 * converged), then [30] tensor-core contraction steps.
 * Synchronous (one device-to-host copy).                                  */
void gp_batched_profile(int on);
int gp_batched_task_stats(const void *d_ws, unsigned long long *h_out);

/* Limit of each dependency wait inside the persistent batched launch (one
 * thread of a CTA spinning on another task's flag), in seconds, for later
 * gp_loglik_grad_batched calls in this process; default 20, accepted range
 * 1e-3 to 600 (else GP_ERR_INVALID).  A wait that runs past it sets that
 * problem's d_info to -1 and makes every CTA leave the launch; problems
 * whose evaluation had finished keep their results, every other problem
 * gets d_info = -1 (if it had no status) and NaN results.  The device stays
 * usable: the next call starts afresh.                                    */
int gp_batched_set_wait_limit(double seconds);

/* Testing aid for the bounded waits (no counterpart in the paper): in later
 * gp_loglik_grad_batched calls of this process, every wait for the Cholesky
 * tile (tile_row, tile_col) of problem `problem` (tile coordinates in that
 * problem's tiles: 64 x 64 in GP_FP64) behaves as if the tile were never
 * produced, so that the first such wait runs into the wait limit.  No GPU
 * fault is involved: the wait ends at its limit like any other.  problem
 * = -1 turns it off.  tile_col > tile_row or a negative index returns
 * GP_ERR_INVALID here; a tile row beyond the problem's tiles makes the
 * batched call return GP_ERR_INVALID before any device work.              */
int gp_batched_test_unset_tile(int problem, int64_t tile_row, int64_t tile_col);

/* Tile policy of the GP_MIXED_F16 batched launch (per device): problems with
 * n <= fp64_max_n run on FP64 64 x 64 tiles (CUDA cores), the others on
 * 128 x 128 tensor-core tiles, in the same launch.  Default 0 (every problem
 * on tensor-core tiles).  gp_batched_autotune chooses it by measurement:
 * it runs the caller's batch (same arguments as gp_loglik_grad_batched,
 * precision GP_MIXED_F16) with each candidate threshold (0 and those of
 * 256, 384, 512, 768, 1024, 1536 below the largest n), one warm-up and two
 * timed launches each, sets the fastest as the policy and returns it in
 * *h_choice; h_ms (nullable, up to 8 entries) receives each candidate's
 * best time in ms, in the order above, and *h_ncand (nullable) their
 * number.  The autotuner synchronises the stream (call it outside a graph
 * capture); the outputs of the last run are left in d_out / d_grad.     */
int gp_batched_set_tile_policy(int64_t fp64_max_n);
/* Host-only check of the batched launch's task order (no device work):
 * rebuilds the merged task list that the launch would run for these sizes
 * (precision GP_FP64 or GP_MIXED_F16, tile threshold fp64_max_n), and
 * returns in *h_ntasks the list length, in *h_bad_order the number of task
 * dependencies that are NOT earlier in the list (0 for a correct plan: the
 * persistent launch cannot deadlock) and in *h_bad_slots the list slots not
 * holding exactly one task (0).                                          */
int gp_batched_plan_check(int nprob, const int64_t *h_n, int precision, int64_t fp64_max_n,
                          int64_t *h_ntasks, int64_t *h_bad_order, int64_t *h_bad_slots);
int64_t gp_batched_tile_policy(void);
int gp_batched_autotune(int nprob, const int64_t *h_n, const double *const *h_dx,
                        const double *const *h_dy, const double *const *h_dmu,
                        const gp_params *h_prm, int precision, void *d_ws, size_t ws_bytes,
                        double *d_out, double *d_grad, int64_t *d_info, void *stream,
                        int64_t *h_choice, double *h_ms, int *h_ncand);

/* Kriging prediction at m new locations (Sec. 1: prediction is the
 * conditional expectation of the latent process given the data, with its
 * variance; Sec. 2.2.2: the Cholesky factor is reused through triangular
 * solves; Sec. 4.3: predictions with standard errors on a grid), from a
 * previous gp_loglik / gp_loglik_grad of the same training data and
 * parameters:
 *   d_x (n x 2) training locations, d_xnew (m x 2) new locations, both
 *   interleaved; d_alpha (n) = C^{-1}(y - mu) as returned by gp_loglik;
 *   mu_new: the (constant) mean at the new locations.
 *   d_mean (m):  mu_new + sum_i K_ij alpha_i,  K_ij = sigma2 k(|x_i - xnew_j| / rho)
 *                (no nugget between a new and a training location: the
 *                prediction is of the latent process).  Matrix-free, FP64
 *                kernel evaluations, compensated sums.
 *   d_var (m, nullable): sigma2 - K_.j^T C^{-1} K_.j = sigma2 - |L^{-1} K_.j|^2
 *                (the variance of the latent process at xnew_j given the
 *                data; its square root is the standard error).  Needs d_L:
 *                the factor as gp_loglik leaves it at the start of its
 *                workspace (n_p x n_p, column-major, lower, ld = ldl >= n_p,
 *                identity padding), and d_ws of gp_predict_workspace_bytes(n,
 *                m, 1) bytes (0 when d_var is NULL: d_L and d_ws may then be
 *                NULL).  FP64 on the CUDA cores: n_p^2 m flops.
 * Non-finite locations set *d_info = -2; after any device-side failure
 * every output is NaN.                                                    */
size_t gp_predict_workspace_bytes(int64_t n, int64_t m, int want_var);
int gp_predict(const double *d_x, int64_t n, const double *d_xnew, int64_t m, const gp_params *prm,
               const double *d_alpha, const double *d_L, int64_t ldl, double mu_new, double *d_mean,
               double *d_var, void *d_ws, size_t ws_bytes, int64_t *d_info, void *stream);

/* ---- simulation (Sec. 1: unconditional realisations and realisations
 * conditional on the data; Sec. 2.3.2: the Cholesky factor times standard
 * normals; Sec. 4.3: posterior realisations on the prediction grid) ------
 *
 * Standard normals: Philox4x64-10 (Salmon et al., SC 2011), a counter-based
 * generator, so every draw is a pure function of its indices.  For
 * realisation c and rows 4q .. 4q+3 the block function of counter
 * (q, c, stream_id, 0) and key (seed, 0) gives four 64-bit words w_k;
 * u_k = ((w_k >> 11) + 1/2) 2^-53 lies in (0, 1); rows 4q, 4q+1 are
 * sqrt(-2 ln u0) (cos, sin)(2 pi u1) and rows 4q+2, 4q+3 the same with
 * (u2, u3) (Box-Muller).  (The paper's package draws with L'Ecuyer's
 * generator; results here are defined by this one.)
 *
 * gp_rng_normal: d_out[i + c ldo] = row i of realisation first + c, for
 * i < n, c < r (column-major n x r, ldo >= n).                            */
int gp_rng_normal(int64_t n, int64_t r, uint64_t seed, uint64_t stream_id, uint64_t first,
                  double *d_out, int64_t ldo, void *stream);

/* Unconditional realisations of N(mu, C) from its factor: column c of d_out
 * (n x r, column-major, ldo >= n) = mu + L e_c, e_c the normals of
 * realisation first + c in stream 0.  d_L: lower factor (ld ldl >= n; its
 * upper part is never read), e.g. the start of a gp_loglik workspace.
 * d_ws: gp_simulate_workspace_bytes(n, r) (the normals).  FP64 on the CUDA
 * cores: n^2 r flops.                                                     */
size_t gp_simulate_workspace_bytes(int64_t n, int64_t r);
int gp_simulate(const double *d_L, int64_t n, int64_t ldl, int64_t r, uint64_t seed, uint64_t first,
                double mu, double *d_out, int64_t ldo, void *d_ws, size_t ws_bytes, void *stream);

/* Realisations of the latent process at m new locations conditional on the
 * data (posterior draws), from a previous gp_loglik of the training data
 * (d_alpha, and d_L = the factor at the start of its workspace, ld ldl >=
 * n_p), with the arguments of gp_predict:
 *   S = K** - K^T C^{-1} K  (the posterior covariance; K** the new
 *       locations' covariance without nugget, K the cross covariance),
 *   S = L* L*^T (unpivoted FP64 Cholesky),
 *   column c of d_out (m x r, ldo >= m) = mean + L* e_c, mean as gp_predict,
 *   e_c the normals of realisation first + c in stream 1.
 * A posterior covariance that is not numerically positive definite (new
 * locations too close to each other or to noise-free data: the failure of
 * Sec. 5) sets *d_info = column + 1 and d_out to NaN.  d_ws:
 * gp_simulate_conditional_workspace_bytes(n, m, r), about 8 (n_p m + m_p^2
 * + m r) bytes.  FP64 on the CUDA cores: n_p^2 m + m^2 n_p + m^3/3 + m^2 r
 * flops.                                                                  */
size_t gp_simulate_conditional_workspace_bytes(int64_t n, int64_t m, int64_t r);
int gp_simulate_conditional(const double *d_x, int64_t n, const double *d_xnew, int64_t m,
                            const gp_params *prm, const double *d_alpha, const double *d_L,
                            int64_t ldl, double mu_new, int64_t r, uint64_t seed, uint64_t first,
                            double *d_out, int64_t ldo, void *d_ws, size_t ws_bytes,
                            int64_t *d_info, void *stream);

/* Log-likelihood without any workspace or allocation (GP_FP64 only).  The
 * paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory when they need a log-likelihood -- code running
 * while a stream is being captured into a CUDA graph, real-time or embedded
 * callers whose device memory is fixed at start-up, plug-ins inside an
 * application that owns every device allocation.  Same arguments and
 * results as gp_loglik with precision GP_FP64, minus the workspace; the
 * caller still passes the inputs and outputs.
 *
 * Scratch: one static device array of GP_NOALLOC_SCRATCH_BYTES (about
 * 2.1 MB) inside libgp, which every GPU that loads the library holds until
 * the process exits.  n above GP_NOALLOC_MAX_N returns GP_ERR_TOO_LARGE
 * before any device work.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture starts.  All calls on a
 * device share the array, which keeps the last call's contents: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Each call rewrites every scratch entry
 * it reads, so earlier calls do not affect its result.                     */
#define GP_NOALLOC_MAX_N 512
#define GP_NOALLOC_SCRATCH_BYTES 2105856
int gp_loglik_noalloc(const double *d_x, const double *d_y, const double *d_mu, int64_t n,
                      const gp_params *prm, double *d_out, double *d_alpha, int64_t *d_info,
                      void *stream);

/* One trailing update of the block Cholesky (Sec. 2.1, the matrix
 * multiplication and subtraction that carries most of the work), on its
 * own:  C -= P P^T on the lower triangle of the m x m block d_C (ldc),
 * with P the m x k block d_P (column-major, ldp).  The tensor-core forms
 * run it on tcgen05 over 16-bit slices (FP32 accumulation, one contraction
 * per 512-deep chunk of k added in FP64); GP_FP64 on the CUDA cores.  d_ws: gp_syrk_workspace_bytes (0 for GP_FP64).  d_info
 * (nullable) receives -1 if a bounded device wait gave up.                */
size_t gp_syrk_workspace_bytes(int64_t m, int64_t k, int precision);
int gp_syrk_lower(double *d_C, int64_t ldc, const double *d_P, int64_t ldp, int64_t m, int64_t k,
                  int precision, void *d_ws, size_t ws_bytes, int64_t *d_info, void *stream);

/* ---- measurement aid ------------------------------------------------ */

/* Number of kernels this library has launched in this process so far. */
int64_t gp_launch_count(void);

/* Kernel classes timed by the optional profiler. */
#define GP_PROF_CONTRACT 0 /* tcgen05 slice contraction (Cholesky update,
                              panel solve, inverse); flops = slice products */
#define GP_PROF_FILL 1     /* covariance fill; bytes = lower-triangle FP64 */
#define GP_PROF_RESIDUAL 2 /* matrix-free refinement residual */
#define GP_PROF_GRAD 3     /* gradient contraction; bytes = lower-triangle FP64 */
#define GP_PROF_DIAG 4     /* tiled Cholesky of a diagonal block (or of the
                              whole matrix in GP_FP64), FP64 with double-float
                              diagonal tiles in GP_MIXED_F16; flops = nb^3/3 */
#define GP_PROF_DIAGINV 5  /* FP64 inverse of a diagonal block; flops = nb^3/3 */
#define GP_PROF_SOLVE 6    /* triangular solves; bytes = 8 per lower entry read */
#define GP_PROF_PACK 7     /* FP64 -> 16-bit slice packing */
#define GP_PROF_FOLD 8     /* double-float pending-update fold into the FP64
                              block column */
/* The contractions of GP_PROF_CONTRACT by role (gp_prof_read of
 * GP_PROF_CONTRACT sums all of them):                                     */
#define GP_PROF_CONTRACT_CHOL 9    /* Cholesky panel solves and trailing updates */
#define GP_PROF_CONTRACT_TRTRI 10  /* blocked inverse of the factor */
#define GP_PROF_CONTRACT_LAUUM 11  /* C^{-1} = X^T X from the inverse factor */

/* gp_prof_enable(1) clears the counters and brackets each later launch of
 * the classes above with a pair of CUDA events recorded on the launch's own
 * stream (host-side only: no device allocation, no synchronisation);
 * gp_prof_enable(0) stops recording.  Not for concurrent use from several
 * host threads.  Returns GP_ERR_CUDA if events cannot be created.        */
int gp_prof_enable(int on);

/* Sums for one class over the launches recorded since gp_prof_enable(1):
 * total event time (ms), launch count, algorithmic flops and bytes.  Waits
 * for the recorded events.  The event pool grows on demand up to 2^20
 * launches; returns GP_ERR_WORKSPACE if any launch since gp_prof_enable(1)
 * went unrecorded (pool cap reached or an event call failed), in which case
 * the sums cover only the recorded launches and must not be used.        */
int gp_prof_read(int cls, double *ms_total, int64_t *launches, double *flops, double *bytes);

/* Launches left unrecorded since gp_prof_enable(1) (0 when the sums of
 * gp_prof_read cover every profiled launch).                              */
int64_t gp_prof_dropped(void);

#ifdef __cplusplus
}
#endif
#endif /* GP_H */
