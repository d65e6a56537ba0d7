// internal.h -- host-side launchers shared between the libgp sources.
#pragma once

#include "common.cuh"

namespace gp {

struct KernParams;

// prof.cu (event timing of selected launches; no-ops unless enabled)
int prof_start(cudaStream_t s);
void prof_stop(int idx, cudaStream_t s, int cls, double flops, double bytes);
// the profiling class of the contractions issued by this host thread (a role
// of GP_PROF_CONTRACT), set for a scope
int prof_contract_class();
struct ProfContractRole {
    int prev;
    explicit ProfContractRole(int cls);
    ~ProfContractRole();
};

// fill.cu
int launch_cov_fill(const double *d_x, int64_t n, int64_t np, const KernParams &kp, double *d_C,
                    int64_t ldc, int64_t *d_info, cudaStream_t s);

// dense_f64.cu
struct F64Mask {
    int out_lower;    // write only entries with row + diag_off >= col
    int64_t diag_off;
    int tri_k;        // op(B)(k, c) vanishes for k < c - tri_off
    int64_t tri_off;
    int64_t kchunk;   // > 0: split K into chunks, accumulate into C with atomics
    int a_lower = 0;  // op(A)(r, k) is read as 0 for k > r (A lower triangular, its
                      // upper part never read)
};
int gemm_f64_ex(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
                int opA, const double *B, int64_t ldb, int opB, double beta, double *C, int64_t ldc,
                int lower, const F64Mask &mask, const int64_t *info, cudaStream_t s);
int gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda, int opA,
             const double *B, int64_t ldb, int opB, double beta, double *C, int64_t ldc, int lower,
             const int64_t *info, cudaStream_t s);
int chol_fp64_tiled(double *A, int64_t ld, int64_t m, int64_t col_base, int64_t *info,
                    cudaStream_t s, bool df_tiles = false);
int trtri_fp64_blocked(const double *L, int64_t ld_l, int64_t m, double *X, int64_t ld_x,
                       double *tmp, const int64_t *info, cudaStream_t s);

// solve.cu
int launch_residual(const double *y, const double *mu, int64_t n, int64_t np, double *r,
                    int64_t *info, cudaStream_t s);
int trsv_blocked(const double *L, int64_t ld, int64_t n, int trans, double *b,
                 const int64_t *info, cudaStream_t s);
int lower_matvec(const double *L, int64_t ld, int64_t n, const double *z, double *y,
                 cudaStream_t s);
int trsv_blocked_skip(const double *L, int64_t ld, int64_t n, int trans, double *b,
                      const int64_t *info, const int *skip, cudaStream_t s);
int launch_loglik_reduce(const double *L, int64_t ld, int64_t n, const double *u, const double *v,
                         const double *resid, double *out, const int64_t *info, cudaStream_t s);

// trsv_persist.cu (single-launch solves; sync holds trsv_sync_ints(n) ints)
size_t trsv_sync_ints(int64_t n);
int trsv_persist(const double *L, int64_t ld, int64_t n, int trans, double *b, int *sync,
                 int64_t *info, const int *skip, cudaStream_t s);

// chol_mixed.cu
size_t chol_mixed_ws_bytes(int64_t np, int S);
// winv (nullable, chol_winv_doubles(np) doubles): receives L_kk^{-1} of every
// 512-column diagonal block (NB x NB each, in block order) for the inverse
size_t chol_winv_doubles(int64_t np);
// outer block width of the mixed factorisation for S slices, and the
// inverse of the 512-column diagonal block at k0 within winv (its ld in *ld)
int64_t chol_block_cols(int S);
const double *winv_block(const double *winv, int64_t np, int S, int64_t k0, int64_t *ld);
// lookahead: run each next diagonal block on the device's side stream while
// the trailing update finishes (off for callers that already run many
// factorisations side by side)
int chol_mixed(double *A, int64_t ld, int64_t np, int S, void *ws, double *winv, int64_t *info,
               cudaStream_t s, bool lookahead = true);
size_t syrk_ws_bytes(int64_t m, int64_t k, int precision, int S);
int syrk_lower(double *C, int64_t ldc, const double *P, int64_t ldp, int64_t m, int64_t k,
               int precision, int S, void *ws, int64_t *info, cudaStream_t s);

// adjoint.cu
size_t grad_ws_bytes(int64_t np, int precision, int S);
int chol_inverse(double *A, int64_t ld, int64_t np, int precision, int S, void *ws,
                 const double *winv, int64_t *info, cudaStream_t s);
int grad_contract(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *W,
                  int64_t ld, const double *alpha, void *ws, int precision, int S, double *grad,
                  const int64_t *info, cudaStream_t s);

// refine.cu
int cov_matvec(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *a,
               double *acc, const int *skip, const int64_t *info, cudaStream_t s);
int refine_alpha(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *L,
                 int64_t ld, const double *r, double *alpha, double *acc, double *s,
                 double *stats, int *conv, int *tsync, int max_evals, double tol, int64_t *info,
                 cudaStream_t st);

// product.cu (the product model: fill, C alpha for the refinement, 4-component gradient)
int prod_fill(const double *d_x, int64_t n, int64_t np, const KernParams &kp, double *d_C,
              int64_t ldc, int64_t *d_info, cudaStream_t s);
int prod_matvec(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *a,
                double *acc, const int *skip, const int64_t *info, cudaStream_t s);
int prod_grad(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *W,
              int64_t ld, const double *alpha, double *part, double *grad, const int64_t *info,
              cudaStream_t s);

// predict.cu (kriging mean and variance at new locations)
size_t predict_ws_bytes(int64_t n, int64_t m, int want_var);
int predict_run(const double *d_x, int64_t n, const double *d_xs, int64_t m, const KernParams &kp,
                const double *d_alpha, const double *d_L, int64_t ldl, double mu_new,
                double *d_mean, double *d_var, void *d_ws, int64_t *d_info, cudaStream_t s);

// simulate.cu (realisations: Philox4x64-10 normals times a triangular factor)
int rng_normals(int64_t n, int64_t rows, int64_t r, uint64_t seed, uint64_t stream, uint64_t first,
                double *out, int64_t ldo, cudaStream_t s);
size_t simulate_ws_bytes(int64_t n, int64_t r);
int simulate_run(const double *d_L, int64_t n, int64_t ldl, int64_t r, uint64_t seed,
                 uint64_t first, double mu, double *d_out, int64_t ldo, void *d_ws, cudaStream_t s);
size_t simulate_cond_ws_bytes(int64_t n, int64_t m, int64_t r);
int simulate_cond_run(const double *d_x, int64_t n, const double *d_xs, int64_t m,
                      const gp_params &prm, const double *d_alpha, const double *d_L, int64_t ldl,
                      double mu_new, int64_t r, uint64_t seed, uint64_t first, double *d_out,
                      int64_t ldo, void *d_ws, int64_t *d_info, cudaStream_t s);

// batch_dag.cu / batch_dag_tc.cu (the batched evaluation as one persistent task-graph launch)
size_t dag_workspace_bytes(int nprob, const int64_t *h_n, int mixed);
int dag_run(int nprob, const int64_t *h_n, const double *const *h_dx, const double *const *h_dy,
            const double *const *h_dmu, const KernParams *kps, int mixed, int64_t fp64_max_n,
            void *d_ws, size_t ws_bytes, double *d_out, double *d_grad, int64_t *d_info,
            cudaStream_t s);
void dag_set_fp64_max_n(int64_t v);
int dag_plan_check(int nprob, const int64_t *h_n, int mixed, int64_t fp64_max_n, int64_t *h_ntasks,
                   int64_t *h_bad_order, int64_t *h_bad_slots);
int64_t dag_fp64_max_n();
int dag_stats(const void *d_ws, unsigned long long *h_out);
void dag_set_profile(int on);
int dag_set_wait_ns(uint64_t ns);
int dag_set_unset_tile(int prob, int64_t i, int64_t j);

}  // namespace gp
