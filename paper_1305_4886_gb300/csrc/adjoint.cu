// adjoint.cu -- the gradient of the log-likelihood (not in the paper; the
// paper's optimiser uses no analytic gradient).
//
// With alpha = C^{-1} r and W = C^{-1}, the adjoint of the log-likelihood
// with respect to C is  Cbar = 1/2 (alpha alpha^T - W),  and
//   d loglik / d theta_j = sum_{i,k} Cbar_ik (dC/dtheta_j)_ik,
// theta = (log sigma2, log rho, log tau2):
//   dC/dlog sigma2 = C - tau2 I,  dC/dlog rho = -sigma2 u k'(u),
//   dC/dlog tau2 = tau2 I.
// W comes from the factor in place: TRTRI (L -> X = L^{-1}) then LAUUM
// (X -> X^T X = C^{-1}, lower), both blocked over 512-row block rows so
// that almost all of their 2n^3/3 flops are contractions that run on the
// same engine as the Cholesky update (tcgen05 BF16 slices in the mixed
// form, FP64 CUDA cores in the FP64 form).  dC/dtheta is recomputed tile by
// tile from the locations inside the contraction kernel and never stored.
//
// Blocked TRTRI, block row k (rows k0..k0+nb), top to bottom:
//   X_kk = L_kk^{-1}                              (FP64, diagonal block)
//   T    = L[k, 0:k0] X[0:k0, 0:k0]                (contraction, X lower)
//   X[k, 0:k0] = -X_kk T                          (contraction)
// Each finished block row of X is packed, transposed, into a store XT
// (XT[j][l] = X[l][j]) that the later TRTRI steps and LAUUM read.
// Blocked LAUUM, block row I:  W[I, 0:I] = sum_{l >= I0} X[l, I]^T X[l, 0:I],
// one contraction over XT per block row, written in place.
#include "internal.h"
#include "kern.cuh"
#include "tc_gemm.h"

namespace gp {

constexpr int64_t GNB = 512;  // block rows of TRTRI / LAUUM

// A packed operand store: [S][rows][kld] 16-bit slices (plus, for three
// slices, the row exponents [rows][kld / 512]), or [rows][kld] FP64.
struct Store {
    void *p = nullptr;
    int *ex = nullptr;
    int64_t rows = 0, kld = 0;
    int f64 = 0;
    int S = 3;
    int64_t kch = TC_CHUNK_K;  // K width of one row bound (three slices: 512 or 1024)
    size_t slice_bytes() const { return (size_t)rows * kld * (f64 ? 8 : 2 * S); }
    size_t ex_bytes() const {
        return (f64 || S != 3) ? 0 : sizeof(int) * (size_t)rows * tc_ex_ld(kld, kch);
    }
};

// FP64 pack: dst[(row_off + r) kld + k_off + k] = op(r, k) (see split_rows).
__global__ void pack_f64_kernel(const double *src, int64_t ld, int64_t R, int64_t K, int64_t Kvalid,
                                int trans, int64_t diag_off, int lower_mask, double *dst,
                                int64_t kld) {
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        int64_t r, k;
        if (trans == 0) { r = r0 + tx; k = k0 + i; }
        else { r = r0 + i; k = k0 + tx; }
        double v = 0.0;
        if (r < R && k < Kvalid) {
            bool zero = lower_mask && (trans ? (k + diag_off < r) : (r + diag_off < k));
            if (!zero) v = trans ? src[k + r * ld] : src[r + k * ld];
        }
        if (trans == 0) t[tx][i] = v; else t[i][tx] = v;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i, k = k0 + tx;
        if (r < R && k < K) dst[r * kld + k] = t[i][tx];
    }
}

static int pack(const Store &st, const double *src, int64_t ld, int64_t R, int64_t K,
                int64_t Kvalid, int trans, int64_t diag_off, int lower_mask, int64_t row_off,
                int64_t k_off, cudaStream_t s) {
    if (R <= 0 || K <= 0) return GP_OK;
    if (row_off + R > st.rows || k_off + K > st.kld) return GP_ERR_INVALID;
    if (st.f64) {
        double *dst = static_cast<double *>(st.p) + row_off * st.kld + k_off;
        dim3 g((unsigned)ceil_div(K, 32), (unsigned)ceil_div(R, 32));
        const int ev = prof_start(s);
        pack_f64_kernel<<<g, 256, 0, s>>>(src, ld, R, K, Kvalid, trans, diag_off, lower_mask, dst,
                                          st.kld);
        GP_LAUNCH_CHECK();
        prof_stop(ev, s, GP_PROF_PACK, 0.0, 16.0 * (double)R * K);
        return GP_OK;
    }
    return split_rows(src, ld, R, K, Kvalid, trans, diag_off, lower_mask, st.S,
                      static_cast<uint16_t *>(st.p), st.ex, st.rows, st.kld, row_off, k_off, s,
                      st.kch);
}

// C (M x N, FP64) = beta C + alpha A[a_row.., a_k..] B[b_row.., b_k..]^T over K.
static int contract(const Store &A, int64_t a_row, int64_t a_k, const Store &B, int64_t b_row,
                    int64_t b_k, int64_t M, int64_t N, int64_t K, double alpha, double beta,
                    double *C, int64_t ldc, int lower, int64_t diag_off, int tri_k,
                    int64_t tri_off, void *acc2, int64_t *info, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return GP_OK;
    if (A.f64) {
        const double *a = static_cast<const double *>(A.p) + a_row * A.kld + a_k;
        const double *b = static_cast<const double *>(B.p) + b_row * B.kld + b_k;
        F64Mask m{lower, diag_off, tri_k, tri_off, 0};
        return gemm_f64_ex(M, N, K, alpha, a, A.kld, 1, b, B.kld, 0, beta, C, ldc, 0, m, info, s);
    }
    TcOperand ta{static_cast<const uint16_t *>(A.p), A.rows, A.kld, A.S, a_row, a_k,
                 A.ex, tc_ex_ld(A.kld, A.kch), A.kch};
    TcOperand tb{static_cast<const uint16_t *>(B.p), B.rows, B.kld, B.S, b_row, b_k,
                 B.ex, tc_ex_ld(B.kld, B.kch), B.kch};
    TcOut o{C, ldc, 0, alpha, beta, lower, diag_off, acc2};
    return tc_gemm(ta, tb, M, N, K, o, tri_k, tri_off, info, s);
}

// lower part of an nb x nb block: dst = src (upper part of dst untouched)
__global__ void copy_lower_kernel(const double *src, int64_t lds, double *dst, int64_t ldd,
                                  int64_t nb, const int64_t *info) {
    if (failed(info)) return;
    const int64_t c = blockIdx.y;
    for (int64_t r = c + threadIdx.x; r < nb; r += blockDim.x) dst[r + c * ldd] = src[r + c * lds];
}

struct GradWs {
    Store XT, SArow, SW, ST;
    double *T = nullptr, *Wd = nullptr, *tmp = nullptr, *part = nullptr;
    void *acc2 = nullptr;  // GNB x np double-float chunk accumulator (tensor path)
    size_t bytes = 0;
};

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

static int64_t ntiles64(int64_t np) {
    const int64_t T = np / TB;
    return T * (T + 1) / 2;
}

static GradWs grad_layout(void *base, int64_t np, int precision, int S) {
    GradWs w;
    char *b = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = a256(off);
        char *p = b ? b + off : nullptr;
        off += bytes;
        return p;
    };
    const int f64 = precision == GP_FP64;
    auto mk = [&](int64_t rows, int64_t kld) {
        Store st;
        st.rows = rows;
        st.kld = kld;
        st.f64 = f64;
        st.S = S;
        st.p = take(st.slice_bytes());
        if (st.ex_bytes()) st.ex = reinterpret_cast<int *>(take(st.ex_bytes()));
        return st;
    };
    const int64_t kldp = round_up(np, 64);
    w.XT = mk(np, kldp);
    w.SArow = mk(GNB, kldp);
    if (!f64 && S == 3) {
        // the inverse's deep contractions (T = L X and X^T X) on 1024-column row
        // bounds: half as many accumulator flushes (the exponent arrays were
        // sized for 512-column chunks, so they have room).  2048 columns were
        // measured too: 0.4% faster over the step and the gradient 3x less
        // accurate (1.1e-6 at n = 16,384), so not kept.
        w.XT.kch = 2 * TC_CHUNK_K;
        w.SArow.kch = 2 * TC_CHUNK_K;
    }
    w.SW = mk(GNB, GNB);
    w.ST = mk(np, GNB);
    w.T = reinterpret_cast<double *>(take(sizeof(double) * GNB * (size_t)np));
    w.Wd = reinterpret_cast<double *>(take(sizeof(double) * GNB * GNB));
    w.tmp = reinterpret_cast<double *>(take(sizeof(double) * TB * GNB));
    // per-tile gradient shares: 3 per tile, 4 for the product model
    w.part = reinterpret_cast<double *>(take(sizeof(double) * 4 * (size_t)ntiles64(np)));
    if (!f64) w.acc2 = take(sizeof(float) * 2 * GNB * (size_t)np);
    w.bytes = a256(off);
    return w;
}

size_t grad_ws_bytes(int64_t np, int precision, int S) {
    return grad_layout(nullptr, np, precision, S).bytes;
}

// In place: A (lower L) -> X = L^{-1} (lower); fills w.XT with X^T.  winv
// (nullable): the diagonal-block inverses the factorisation already formed
// (GNB x GNB each, in block order), used instead of recomputing them.
static int trtri_inplace(double *A, int64_t ld, int64_t np, GradWs &w, const double *winv,
                         int64_t *info, cudaStream_t s) {
    for (int64_t k0 = 0; k0 < np; k0 += GNB) {
        const int64_t nb = (np - k0) < GNB ? (np - k0) : GNB;
        double *Akk = A + k0 + k0 * ld;
        const double *Wd = w.Wd;
        int64_t wld = nb;
        if (winv) {
            Wd = winv_block(winv, np, w.XT.S, k0, &wld);
        } else {
            const int ev = prof_start(s);
            GP_TRY(trtri_fp64_blocked(Akk, ld, nb, w.Wd, nb, w.tmp, info, s));
            prof_stop(ev, s, GP_PROF_DIAGINV, (double)nb * nb * nb / 3.0, 0.0);
        }
        if (k0 > 0) {
            // T (nb x k0) = L[k, 0:k0] X[0:k0, 0:k0]
            GP_TRY(pack(w.SArow, A + k0, ld, nb, k0, k0, 0, 0, 0, 0, 0, s));
            GP_TRY(contract(w.SArow, 0, 0, w.XT, 0, 0, nb, k0, k0, 1.0, 0.0, w.T, nb, 0, 0, 1, 0,
                            w.acc2, info, s));
            // X[k, 0:k0] = -X_kk T
            GP_TRY(pack(w.SW, Wd, wld, nb, nb, nb, 0, 0, 1, 0, 0, s));
            GP_TRY(pack(w.ST, w.T, nb, k0, nb, nb, 1, 0, 0, 0, 0, s));
            GP_TRY(contract(w.SW, 0, 0, w.ST, 0, 0, nb, k0, nb, -1.0, 0.0, A + k0, ld, 0, 0, 0, 0,
                            w.acc2, info, s));
        }
        copy_lower_kernel<<<dim3(1, (unsigned)nb), 256, 0, s>>>(Wd, wld, Akk, ld, nb, info);
        GP_LAUNCH_CHECK();
        // XT[j][l] = X[l][j] for l in block k, j < k0 + nb (zero above the
        // diagonal).  With 1024-column row bounds a block that completes a
        // chunk packs the chunk's two blocks together (one bound over both);
        // a block that opens one packs itself, bounded over its own columns,
        // which is what the next block's T = L X reads of the open chunk.
        const int64_t kc = w.XT.kch;
        const int64_t c0 = (k0 / kc) * kc;
        GP_TRY(pack(w.XT, A + c0, ld, k0 + nb, k0 + nb - c0, k0 + nb - c0, 1, c0, 1, 0, c0, s));
    }
    return GP_OK;
}

// In place: A (lower X) -> W = X^T X (lower), reading X from w.XT.  Each
// block row's K range starts at its chunk boundary (with 1024-column row
// bounds below i0; the extra columns l < i0 multiply X(l, i0 + r) = 0).
static int lauum_inplace(double *A, int64_t ld, int64_t np, GradWs &w, int64_t *info,
                         cudaStream_t s) {
    const Store &X = w.XT;
    for (int64_t i0 = 0; i0 < np; i0 += GNB) {
        const int64_t nb = (np - i0) < GNB ? (np - i0) : GNB;
        const int64_t k0 = (i0 / X.kch) * X.kch;
        GP_TRY(contract(X, i0, k0, X, 0, k0, nb, i0 + nb, np - k0, 1.0, 0.0, A + i0, ld, 1, i0, 0,
                        0, w.acc2, info, s));
    }
    return GP_OK;
}

int chol_inverse(double *A, int64_t ld, int64_t np, int precision, int S, void *ws,
                 const double *winv, int64_t *info, cudaStream_t s) {
    GradWs w = grad_layout(ws, np, precision, S);
    {
        ProfContractRole role(GP_PROF_CONTRACT_TRTRI);
        GP_TRY(trtri_inplace(A, ld, np, w, winv, info, s));
    }
    ProfContractRole role(GP_PROF_CONTRACT_LAUUM);
    GP_TRY(lauum_inplace(A, ld, np, w, info, s));
    return GP_OK;
}

// ---------------------------------------------------------------------------
// Gradient contraction over the lower 64 x 64 tiles of W (FP64):
//   g0 = sum_{i>k} (a_i a_k - W_ik) C_ik + sum_i Cbar_ii sigma2
//   g1 = sum_{i>k} (a_i a_k - W_ik) dC_ik/dlog rho
//   g2 = tau2 sum_i Cbar_ii,          Cbar_ii = (a_i^2 - W_ii) / 2
// (the off-diagonal pairs counted twice through the factor 2 Cbar_ik).
// One partial triple per tile; a single CTA sums them in tile order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) grad_contract_kernel(const double2 *__restrict__ x, int64_t n,
                                                            KernParams kp, const double *W,
                                                            int64_t ld, const double *a,
                                                            double *part, const int64_t *info) {
    __shared__ double2 xc[TB];
    __shared__ double tab[EXP_TAB];
    stage_exp_table(kp, tab);
    __shared__ double ac[TB];
    __shared__ double red[3][8];
    if (failed(info)) return;
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    const int tid = threadIdx.x;
    if (tid < TB) {
        const int64_t j = col0 + tid;
        xc[tid] = (j < n) ? x[j] : make_double2(0.0, 0.0);
        ac[tid] = (j < n) ? a[j] : 0.0;
    }
    __syncthreads();
    const int r = tid & (TB - 1), cg = tid >> 6;
    const int64_t i = row0 + r;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (i < n) {
        const double2 xi = x[i];
        const double ai = a[i];
        for (int c = cg; c < TB; c += 4) {
            const int64_t k = col0 + c;
            if (k >= n || k > i) continue;
            const double w = W[i + k * ld];
            if (k == i) {
                const double cb = 0.5 * (ai * ai - w);
                g0 = fma(cb, kp.s2, g0);
                g2 = fma(cb, kp.tau2, g2);
            } else {
                const double cb2 = fma(ai, ac[c], -w);
                double cv, dr;
                cov_and_dlogrho(kp, pair_dist(xi, xc[c]), cv, dr, tab);
                g0 = fma(cb2, cv, g0);
                g1 = fma(cb2, dr, g1);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
        g1 += __shfl_xor_sync(0xffffffffu, g1, o);
        g2 += __shfl_xor_sync(0xffffffffu, g2, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = g0;
        red[1][tid >> 5] = g1;
        red[2][tid >> 5] = g2;
    }
    __syncthreads();
    if (tid < 3) {
        double sum = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) sum += red[tid][w8];
        part[3 * (int64_t)blockIdx.x + tid] = sum;
    }
}

// The same contraction with C, dC/dlog rho and the weights a_i a_k - W_ik
// in double-float on the FP32 pipe (tensor-core forms); W is split into
// (hi, lo) by integer operations and the diagonal terms stay in FP64.
__global__ void __launch_bounds__(256) grad_contract_df_kernel(const double2 *__restrict__ x,
                                                               int64_t n, KernParams kp,
                                                               const double *W, int64_t ld,
                                                               const double *a, double *part,
                                                               const int64_t *info) {
    __shared__ float4 xc[TB];
    __shared__ float2 tab[DF_TAB];
    __shared__ float2 ac[TB];
    __shared__ double red[3][8];
    stage_df_table(kp.kd, tab);
    if (failed(info)) return;
    int64_t ti, tj;
    lower_tile_coords(blockIdx.x, ti, tj);
    const int64_t row0 = ti * TB, col0 = tj * TB;
    const int tid = threadIdx.x;
    if (tid < TB) {
        const int64_t j = col0 + tid;
        xc[tid] = df_point(j < n ? x[j] : make_double2(0.0, 0.0));
        const dfl aj =
            f64_to_df(static_cast<unsigned long long>(__double_as_longlong(j < n ? a[j] : 0.0)));
        ac[tid] = make_float2(aj.h, aj.l);
    }
    __syncthreads();
    const int r = tid & (TB - 1), cg = tid >> 6;
    const int64_t i = row0 + r;
    double g0 = 0.0, g2 = 0.0;
    dfl h0{0.0f, 0.0f}, h1{0.0f, 0.0f};
    if (i < n) {
        const float4 xi = df_point(x[i]);
        const double ai = a[i];
        const dfl aid = f64_to_df(static_cast<unsigned long long>(__double_as_longlong(ai)));
        for (int c = cg; c < TB; c += 4) {
            const int64_t k = col0 + c;
            if (k >= n || k > i) continue;
            const double w = W[i + k * ld];
            if (k == i) {
                const double cb = 0.5 * (ai * ai - w);
                g0 = fma(cb, kp.s2, g0);
                g2 = fma(cb, kp.tau2, g2);
            } else {
                const dfl wd = f64_to_df(static_cast<unsigned long long>(__double_as_longlong(w)));
                const dfl cb2 = df_add(df_mul(aid, dfl{ac[c].x, ac[c].y}), df_neg(wd));
                dfl cv, dr;
                df_cov<true>(kp.kind, kp.kd, df_dist(xi, xc[c]), tab, cv, dr);
                h0 = df_add(h0, df_mul(cb2, cv));
                h1 = df_add(h1, df_mul(cb2, dr));
            }
        }
    }
    g0 += df_to_double(h0);
    double g1 = df_to_double(h1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
        g1 += __shfl_xor_sync(0xffffffffu, g1, o);
        g2 += __shfl_xor_sync(0xffffffffu, g2, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = g0;
        red[1][tid >> 5] = g1;
        red[2][tid >> 5] = g2;
    }
    __syncthreads();
    if (tid < 3) {
        double sum = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) sum += red[tid][w8];
        part[3 * (int64_t)blockIdx.x + tid] = sum;
    }
}

__global__ void __launch_bounds__(1024) grad_reduce_kernel(const double *part, int64_t ntiles,
                                                           double *grad, const int64_t *info) {
    __shared__ double ps[3][1024];
    double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
    for (int64_t t = threadIdx.x; t < ntiles; t += 1024) {
        for (int q = 0; q < 3; ++q) {  // Neumaier
            const double x = part[3 * t + q], u = s[q] + x;
            c[q] += (fabs(s[q]) >= fabs(x)) ? (s[q] - u) + x : (x - u) + s[q];
            s[q] = u;
        }
    }
    for (int q = 0; q < 3; ++q) ps[q][threadIdx.x] = s[q] + c[q];
    __syncthreads();
    if (threadIdx.x < 3) {
        const int q = threadIdx.x;
        double S = 0.0, Cc = 0.0;
        for (int t = 0; t < 1024; ++t) {
            const double x = ps[q][t], u = S + x;
            Cc += (fabs(S) >= fabs(x)) ? (S - u) + x : (x - u) + S;
            S = u;
        }
        grad[q] = (*info != 0) ? nan("") : S + Cc;
    }
}

int grad_contract(const double *d_x, int64_t n, int64_t np, const KernParams &kp, const double *W,
                  int64_t ld, const double *alpha, void *ws, int precision, int S, double *grad,
                  const int64_t *info, cudaStream_t s) {
    GradWs w = grad_layout(ws, np, precision, S);
    if (kp.product) return prod_grad(d_x, n, np, kp, W, ld, alpha, w.part, grad, info, s);
    const int64_t nt = ntiles64(np);
    const int ev = prof_start(s);
    if (kp.use_df)
        grad_contract_df_kernel<<<(unsigned)nt, 256, 0, s>>>(reinterpret_cast<const double2 *>(d_x),
                                                              n, kp, W, ld, alpha, w.part, info);
    else
        grad_contract_kernel<<<(unsigned)nt, 256, 0, s>>>(reinterpret_cast<const double2 *>(d_x), n,
                                                           kp, W, ld, alpha, w.part, info);
    GP_LAUNCH_CHECK();
    prof_stop(ev, s, GP_PROF_GRAD, 0.0, 8.0 * (double)np * (double)(np + 1) / 2.0);
    grad_reduce_kernel<<<1, 1024, 0, s>>>(w.part, nt, grad, info);
    GP_LAUNCH_CHECK();
    return GP_OK;
}

}  // namespace gp
