// internal.h -- host-side launchers shared between the libgp sources.
#pragma once

#include "common.cuh"

namespace gp {

struct KernParams;

// fill.cu
int launch_cov_fill(const double *d_x, int64_t n, int64_t np, const KernParams &kp, double *d_C,
                    int64_t ldc, int64_t *d_info, cudaStream_t s);

// dense_f64.cu
int gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda, int opA,
             const double *B, int64_t ldb, int opB, double beta, double *C, int64_t ldc, int lower,
             const int64_t *info, cudaStream_t s);
int chol_fp64_tiled(double *A, int64_t ld, int64_t m, int64_t col_base, int64_t *info,
                    cudaStream_t s);
int trtri_fp64_blocked(const double *L, int64_t ld_l, int64_t m, double *X, int64_t ld_x,
                       double *tmp, const int64_t *info, cudaStream_t s);

// solve.cu
int launch_residual(const double *y, const double *mu, int64_t n, int64_t np, double *r,
                    int64_t *info, cudaStream_t s);
int trsv_blocked(const double *L, int64_t ld, int64_t n, int trans, double *b,
                 const int64_t *info, cudaStream_t s);
int lower_matvec(const double *L, int64_t ld, int64_t n, const double *z, double *y,
                 cudaStream_t s);
int launch_loglik_reduce(const double *L, int64_t ld, int64_t n, const double *v, double *out,
                         const int64_t *info, cudaStream_t s);

}  // namespace gp
