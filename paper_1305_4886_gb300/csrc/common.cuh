// common.cuh -- shared definitions of the libgp CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gp.h"

namespace gp {

constexpr int TB = 64;        // FP64 CUDA-core tile (diagonal POTRF / TRSM / TRSV)
constexpr int PAD = GP_PAD;   // padding granularity of n

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// The first device-side failure wins: d_info is only written while it is 0.
__device__ __forceinline__ void set_info(int64_t *info, int64_t v) {
    atomicCAS(reinterpret_cast<unsigned long long *>(info), 0ull,
              static_cast<unsigned long long>(v));
}

__device__ __forceinline__ bool failed(const int64_t *info) {
    return *reinterpret_cast<const volatile int64_t *>(info) != 0;
}

// Entry e of the lower triangle {(r, c): c <= r < n} of an n x n tile with the
// columns in DESCENDING order (column n-1 first, rows ascending within a
// column): the trailing triangle of elimination step j is then the prefix
// e < (n-1-j)(n-j)/2.  For e below 2^20 (the float square root is exact
// enough, and the two guards fix its last unit).
__device__ __forceinline__ void tri_desc_entry(int e, int n, int &r, int &c) {
    int t = static_cast<int>((sqrtf(8.0f * static_cast<float>(e) + 1.0f) - 1.0f) * 0.5f);
    if ((t + 1) * (t + 2) / 2 <= e) ++t;
    if (t * (t + 1) / 2 > e) --t;
    c = n - 1 - t;
    r = c + (e - t * (t + 1) / 2);
}

// Map a linear index over the lower-triangular tile grid to (ti, tj), ti >= tj.
__device__ __forceinline__ void lower_tile_coords(int64_t t, int64_t &ti, int64_t &tj) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    ti = i;
    tj = t - i * (i + 1) / 2;
}

}  // namespace gp

namespace gp {
void count_launch();  // api.cu: tally of this library's kernel launches
}

// Every kernel launch in libgp is followed by this check, which also counts it.
#define GP_LAUNCH_CHECK()                                   \
    do {                                                    \
        gp::count_launch();                                 \
        cudaError_t e_ = cudaGetLastError();                \
        if (e_ != cudaSuccess) return GP_ERR_CUDA;          \
    } while (0)

#define GP_TRY(expr)                                        \
    do {                                                    \
        int s_ = (expr);                                    \
        if (s_ != GP_OK) return s_;                         \
    } while (0)
