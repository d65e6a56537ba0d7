// kern_df.cuh -- the covariance function in double-float arithmetic on the
// FP32 pipe, for the tensor-core forms.
//
// The fill, the matrix-free residual and the gradient contraction evaluate
// sigma2 k(d / rho) (and its log-rho derivative) once per pair: about 26
// FP64 operations each, on a part whose FP64 pipe runs at 1/64 of its FP32
// rate.  Here a value is an unevaluated pair (h, l) of FP32 numbers with
// |l| <= ulp(h) / 2, about 48 significant bits, combined with the
// error-free transformations two_sum (Knuth) and two_prod (an FMA gives the
// product's rounding error exactly); the add / multiply / square-root
// compositions follow Dekker (1971) and the double-double library of Hida,
// Li and Bailey (2001).  Every FP32 operation goes through an _rn intrinsic
// so that the compiler neither contracts nor reorders it.
//
// Accuracy: distances and the exponent argument a carry about 2^-46 relative
// error and exp(-a) about 2^-46 + a 2^-47, i.e. a few hundred FP64 ulps: far
// below the 2^-32 operand slices of the mixed form and below what the
// FP64-grade form's 1e-12 log-likelihood agreement needs.  exp(-a) flushes
// to zero beyond a = 87 (below 2^-125), an absolute change of at most
// (1 + a + a^2/3) 2^-125 sigma2 <= 1e-33 sigma2 per entry.
//
// exp(-a) is table driven (Tang's method, with a finer table): with
// k = round(256 a / ln 2) = 256 m + j and r = a - k ln2/256
// (|r| <= ln2/512, ln2/256 carried in three parts so that the reduction
// error stays near 2^-63 absolute for k < 2^15),
//     exp(-a) = 2^-m 2^(-j/256) exp(-r),
// exp(-r) = 1 - r + r^2/2 - r^3/6 + r^4/24 (the r^5 term is below 4e-17),
// the first three terms in double-float and the last two in FP32, and the
// 256 values 2^(-j/256) as double-float pairs computed on the host in
// extended precision.
#pragma once

#include <math.h>

#include "common.cuh"

namespace gp {

constexpr int DF_TAB = 256;

struct dfl {
    float h, l;
};

// s + e = a + b exactly.
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ dfl df_quick_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a b exactly (barring underflow).
__device__ __forceinline__ dfl df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = df_two_sum(a.h, b.h);
    const dfl t = df_two_sum(a.l, b.l);
    s = df_quick_sum(s.h, __fadd_rn(s.l, t.h));
    return df_quick_sum(s.h, __fadd_rn(s.l, t.l));
}

__device__ __forceinline__ dfl df_add_f(dfl a, float b) {
    const dfl s = df_two_sum(a.h, b);
    return df_quick_sum(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    dfl p = df_two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, p.l);
    p.l = __fmaf_rn(a.l, b.h, p.l);
    return df_quick_sum(p.h, p.l);
}

__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
    dfl p = df_two_prod(a.h, b);
    p.l = __fmaf_rn(a.l, b, p.l);
    return df_quick_sum(p.h, p.l);
}

__device__ __forceinline__ dfl df_sqr(dfl a) {
    dfl p = df_two_prod(a.h, a.h);
    p.l = __fmaf_rn(__fmul_rn(2.0f, a.h), a.l, p.l);
    return df_quick_sum(p.h, p.l);
}

// 1 / a for a != 0: an FP32 reciprocal refined by one Newton step,
// y + y (1 - a y), with the residual 1 - a y formed in double-float (the
// FP32 seed's relative error 2^-23 squares to below the pair's precision).
__device__ __forceinline__ dfl df_rcp(dfl a) {
    const float y = __frcp_rn(a.h);
    dfl p = df_two_prod(a.h, y);  // a.h y exactly
    p.l = __fmaf_rn(a.l, y, p.l);
    const dfl e = df_add_f({-p.h, -p.l}, 1.0f);  // 1 - a y
    return df_add_f(df_mul_f(e, y), y);
}

// a - b c
__device__ __forceinline__ dfl df_fms(dfl a, dfl b, dfl c) { return df_add(a, df_neg(df_mul(b, c))); }

// sqrt of a >= 0: an FP32 root refined once against the double-float
// residual (a - s^2 is exact through the FMA to FP32 precision).
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    if (!(a.h > 0.0f)) return {0.0f, 0.0f};
    float y = rsqrtf(a.h);
    y = __fmul_rn(y, __fmaf_rn(__fmul_rn(-0.5f, a.h), __fmul_rn(y, y), 1.5f));  // 1/sqrt to FP32
    const float s = __fmul_rn(a.h, y);
    const float res = __fadd_rn(__fmaf_rn(-s, s, a.h), a.l);
    return df_quick_sum(s, __fmul_rn(res, __fmul_rn(0.5f, y)));
}

// Euclidean distance of two points (coordinate differences first).
__device__ __forceinline__ dfl df_dist(float4 p, float4 q) {
    dfl dx = df_two_sum(p.x, -q.x);
    dx = df_two_sum(dx.h, __fadd_rn(dx.l, __fsub_rn(p.y, q.y)));
    dfl dy = df_two_sum(p.z, -q.z);
    dy = df_two_sum(dy.h, __fadd_rn(dy.l, __fsub_rn(p.w, q.w)));
    const dfl sx = df_sqr(dx), sy = df_sqr(dy);
    // both squares are >= 0: no cancellation in their sum
    const dfl s = df_two_sum(sx.h, sy.h);
    return df_sqrt(df_quick_sum(s.h, __fadd_rn(s.l, __fadd_rn(sx.l, sy.l))));
}

// Parameters of the double-float evaluation (set on the host).
struct KernDf {
    dfl scale;           // sqrt(2 nu) / rho
    dfl s2;              // sigma2
    dfl diag;            // sigma2 + tau2
    float2 tab[DF_TAB];  // 2^(-j/256) as (hi, lo)
};

// exp(-a) for a >= 0; tab in shared memory.
__device__ __forceinline__ dfl df_exp_neg(dfl a, const float2 *tab) {
    constexpr float INV_L = 369.32992553710938f;          // 256 / ln 2 (FP32)
    constexpr float C1 = 0.00270843505859375f;             // 355 2^-17 (9 bits: k C1 exact)
    constexpr float C2 = -8.288845378956466e-07f;          // next 24 bits of ln2/256
    constexpr float C3 = 6.432011600578363e-15f;           // next 24 bits
    if (!(a.h < 87.0f)) return {0.0f, 0.0f};               // below 2^-125 (or NaN input)
    const float kf = rintf(__fmul_rn(a.h, INV_L));
    const int k = static_cast<int>(kf);
    // r = a - k (C1 + C2 + C3); a.h - k C1 is exact
    dfl r = df_two_sum(__fmaf_rn(-kf, C1, a.h), a.l);
    r = df_add(r, df_neg(df_two_prod(kf, C2)));
    r = df_add_f(r, __fmul_rn(-kf, C3));
    // exp(-r) = (1 - r + r^2/2) - (r^3/6 - r^4/24)
    const dfl q = df_sqr(r);
    dfl e = df_add(df_add_f(df_neg(r), 1.0f), dfl{__fmul_rn(0.5f, q.h), __fmul_rn(0.5f, q.l)});
    const float r3 = __fmul_rn(__fmul_rn(r.h, r.h), r.h);
    e = df_add_f(e, -__fmul_rn(r3, __fmaf_rn(-r.h, 1.0f / 24.0f, 1.0f / 6.0f)));
    const float2 t = tab[k & (DF_TAB - 1)];
    e = df_mul(e, dfl{t.x, t.y});
    // 2^-m, m = k / 256 <= 125: exact scaling of both parts
    const float sc = __int_as_float((127 - (k >> 8)) << 23);
    return {__fmul_rn(e.h, sc), __fmul_rn(e.l, sc)};
}

// sigma2 k(a) for a distinct pair with a = scale d, and the log-rho
// derivative -sigma2 a k'(a):
//   exp: s2 e^-a, s2 a e^-a;  Matern 3/2: s2 (1+a) e^-a, s2 a^2 e^-a;
//   Matern 5/2: s2 (1+a+a^2/3) e^-a, s2 a^2 (1+a)/3 e^-a.
template <bool WANT_DR>
__device__ __forceinline__ void df_cov_s(int kind, dfl scale, dfl s2, dfl d, const float2 *tab,
                                         dfl &c, dfl &dr) {
    const dfl a = df_mul(d, scale);
    const dfl e = df_mul(df_exp_neg(a, tab), s2);
    if (kind == GP_KERNEL_EXP) {
        c = e;
        if (WANT_DR) dr = df_mul(e, a);
    } else if (kind == GP_KERNEL_MATERN32) {
        c = df_mul(df_add_f(a, 1.0f), e);
        if (WANT_DR) dr = df_mul(df_sqr(a), e);
    } else {
        constexpr dfl THIRD{0.3333333432674408f, -9.934107758624577e-09f};
        const dfl a2_3 = df_mul(df_sqr(a), THIRD);
        const dfl p = df_add_f(a, 1.0f);
        c = df_mul(df_add(p, a2_3), e);
        if (WANT_DR) dr = df_mul(df_mul(a2_3, p), e);
    }
}

template <bool WANT_DR>
__device__ __forceinline__ void df_cov(int kind, const KernDf &kd, dfl d, const float2 *tab,
                                       dfl &c, dfl &dr) {
    df_cov_s<WANT_DR>(kind, kd.scale, kd.s2, d, tab, c, dr);
}

// FP64 x = hi + lo with integer operations only (no FP64 pipe): hi keeps
// the top 24 significant bits (truncated), lo the remaining 29 rounded to
// FP32.  Magnitudes below 2^-126 map to 0 and lo parts below 2^-126 are
// dropped.
__device__ __forceinline__ dfl f64_to_df(unsigned long long u) {
    const unsigned int sign = static_cast<unsigned int>(u >> 32) & 0x80000000u;
    const int E = static_cast<int>((u >> 52) & 0x7FF);
    const int ef = E - 1023 + 127;
    dfl r{0.0f, 0.0f};
    if (E == 0 || ef <= 0) return r;
    if (ef >= 255) {
        r.h = __int_as_float(sign | 0x7F800000u);
        return r;
    }
    const unsigned long long mant = u & 0x000FFFFFFFFFFFFFull;
    r.h = __int_as_float(sign | (static_cast<unsigned int>(ef) << 23) |
                         static_cast<unsigned int>(mant >> 29));
    const int es = E - 1075;  // weight of the mantissa's last bit
    if (es >= -126) {
        const float lf = __uint2float_rn(static_cast<unsigned int>(mant & 0x1FFFFFFFull));
        r.l = __int_as_float(__float_as_int(lf * __int_as_float((es + 127) << 23)) | sign);
    }
    return r;
}

// FP32 -> FP64 by rewriting the bits, with integer operations only (no FP64
// pipe, which runs at 1/64 of the FP32 rate here): zeros, subnormals
// (m 2^-149 with the leading bit of m at position p: exponent p - 149,
// fraction m shifted up by 52 - p) and normal numbers (finite inputs).
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned long long sgn = static_cast<unsigned long long>(u & 0x80000000u) << 32;
    const unsigned int e = (u >> 23) & 0xFFu;
    const unsigned int m = u & 0x7FFFFFu;
    unsigned long long bits;
    if (e != 0) {
        bits = (static_cast<unsigned long long>(e + 896u) << 52) |
               (static_cast<unsigned long long>(m) << 29);
    } else if (m != 0) {
        const int p = 31 - __clz(static_cast<int>(m));
        bits = (static_cast<unsigned long long>(p + 874) << 52) |
               ((static_cast<unsigned long long>(m) << (52 - p)) & 0xFFFFFFFFFFFFFull);
    } else {
        bits = 0ull;
    }
    return __longlong_as_double(static_cast<long long>(sgn | bits));
}

// f 2^k in FP64 by integer operations: the conversion above with k added to
// the exponent field (exact while the result stays a normal FP64 number,
// which holds for |k| <= 800 and finite f).
__device__ __forceinline__ double f32_to_f64_scaled(float f, int k) {
    const long long b = __double_as_longlong(f32_to_f64(f));
    if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return __longlong_as_double(b);
    return __longlong_as_double(b + (static_cast<long long>(k) << 52));
}

// hi + lo in FP64 (one FP64 add).
__device__ __forceinline__ double df_to_double(dfl a) { return f32_to_f64(a.h) + f32_to_f64(a.l); }

// A point's coordinates as double-float pairs (x_h, x_l, y_h, y_l), by
// integer operations (a coordinate to about 2^-48 of its magnitude).
__device__ __forceinline__ float4 df_point(double2 p) {
    const dfl x = f64_to_df(static_cast<unsigned long long>(__double_as_longlong(p.x)));
    const dfl y = f64_to_df(static_cast<unsigned long long>(__double_as_longlong(p.y)));
    return make_float4(x.h, x.l, y.h, y.l);
}

// Stage the table in shared memory (call before the CTA's first barrier).
__device__ __forceinline__ void stage_df_table(const KernDf &kd, float2 *tab) {
    for (int j = threadIdx.x; j < DF_TAB; j += blockDim.x) tab[j] = kd.tab[j];
}

inline KernDf make_kern_df(const gp_params &p) {
    KernDf k;
    double c = 1.0;
    if (p.kernel == GP_KERNEL_MATERN32) c = 1.7320508075688772;  // sqrt(3)
    if (p.kernel == GP_KERNEL_MATERN52) c = 2.2360679774997897;  // sqrt(5)
    const double sc = c / p.rho;
    const float sh = static_cast<float>(sc), s2h = static_cast<float>(p.sigma2);
    k.scale = {sh, static_cast<float>(sc - static_cast<double>(sh))};
    k.s2 = {s2h, static_cast<float>(p.sigma2 - static_cast<double>(s2h))};
    const double dg = p.sigma2 + p.tau2;
    const float dgh = static_cast<float>(dg);
    k.diag = {dgh, static_cast<float>(dg - static_cast<double>(dgh))};
    for (int j = 0; j < DF_TAB; ++j) {
        const long double v = exp2l(-static_cast<long double>(j) / DF_TAB);
        const float h = static_cast<float>(v);
        k.tab[j] = make_float2(h, static_cast<float>(v - static_cast<long double>(h)));
    }
    return k;
}

}  // namespace gp
