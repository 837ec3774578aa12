// gwns_df.cuh -- double-float arithmetic: a value held as the unevaluated sum
// h + l of two floats (|l| <= ulp(h)/2), about 48 significant bits, computed
// on the FP32 pipe. On GB300 the FP64 pipe issues one warp instruction per 64
// cycles per sub-partition, the FP32 pipe one per cycle, so the per-point
// coefficient stage of the mixed form runs in double-float.
//
// The building blocks are the error-free transformations of Dekker (1971) and
// Knuth (TAOCP vol. 2): TwoSum, FastTwoSum and the FMA-based TwoProd; the
// sums are the "sloppy" double-float sums (error about 2^-48 of the operands'
// magnitudes, which is what the operands themselves carry). The transcendental
// functions reduce their argument against a table point or a multiple of pi/2
// and finish with a short polynomial, with only the leading terms in
// double-float; each states its range and accuracy.
//
// Plain C++ besides the qualifiers, so the same code compiles for the host
// (where a CPU test checks it against 60-digit references) and for sm_103a.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "gwns_tables.cuh"

#if defined(__CUDACC__)
#define DFI __host__ __device__ __forceinline__
#define DFD __device__ __forceinline__      // reads the device tables
#else
#define DFI static inline
#define DFD static inline
#endif

namespace gwns {

struct dfl {
    float h, l;
};

// Single roundings that the compiler must not contract into an FMA.
#if defined(__CUDA_ARCH__)
DFI float f_add(float a, float b) { return __fadd_rn(a, b); }
DFI float f_sub(float a, float b) { return __fsub_rn(a, b); }
DFI float f_mul(float a, float b) { return __fmul_rn(a, b); }
DFI float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
DFI float f_rcp(float a) { return __frcp_rn(a); }
DFI float f_sqrt(float a) { return __fsqrt_rn(a); }
DFI float f_rint(float a) { return rintf(a); }
DFI float i_as_f(int32_t i) { return __int_as_float(i); }
DFI int32_t f_as_i(float f) { return __float_as_int(f); }
#else
DFI float f_add(float a, float b) { return a + b; }
DFI float f_sub(float a, float b) { return a - b; }
DFI float f_mul(float a, float b) { return a * b; }
DFI float f_fma(float a, float b, float c) { return fmaf(a, b, c); }
DFI float f_rcp(float a) { return 1.0f / a; }
DFI float f_sqrt(float a) { return sqrtf(a); }
DFI float f_rint(float a) { return rintf(a); }
DFI float i_as_f(int32_t i) { float f; memcpy(&f, &i, 4); return f; }
DFI int32_t f_as_i(float f) { int32_t i; memcpy(&i, &f, 4); return i; }
#endif

// A double constant as a double-float (folded at compile time).
#define DFC(x) (::gwns::dfl{(float)(x), (float)((x) - (double)(float)(x))})

// ------------------------------------------------- error-free transformations
DFI dfl two_sum_f(float a, float b) {
    const float s = f_add(a, b);
    const float bb = f_sub(s, a);
    return dfl{s, f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb))};
}
// |a| >= |b| (or a == 0)
DFI dfl fast_two_sum_f(float a, float b) {
    const float s = f_add(a, b);
    return dfl{s, f_sub(b, f_sub(s, a))};
}

// ------------------------------------------------------------- arithmetic
DFI dfl df_neg(dfl x) { return dfl{-x.h, -x.l}; }
DFI dfl df_add(dfl x, dfl y) {
    const dfl s = two_sum_f(x.h, y.h);
    return fast_two_sum_f(s.h, f_add(s.l, f_add(x.l, y.l)));
}
DFI dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
DFI dfl df_add_f(dfl x, float b) {
    const dfl s = two_sum_f(x.h, b);
    return fast_two_sum_f(s.h, f_add(s.l, x.l));
}
DFI dfl df_mul(dfl x, dfl y) {
    const float p = f_mul(x.h, y.h);
    float e = f_fma(x.h, y.h, -p);
    e = f_fma(x.h, y.l, e);
    e = f_fma(x.l, y.h, e);
    return fast_two_sum_f(p, e);
}
DFI dfl df_mul_f(dfl x, float b) {
    const float p = f_mul(x.h, b);
    float e = f_fma(x.h, b, -p);
    e = f_fma(x.l, b, e);
    return fast_two_sum_f(p, e);
}
DFI dfl df_sqr(dfl x) {
    const float p = f_mul(x.h, x.h);
    float e = f_fma(x.h, x.h, -p);
    e = f_fma(f_add(x.h, x.h), x.l, e);
    return fast_two_sum_f(p, e);
}
// x * 2^k for a power of two p2 = 2^k (exact without underflow)
DFI dfl df_scale(dfl x, float p2) { return dfl{f_mul(x.h, p2), f_mul(x.l, p2)}; }
DFI double df_to_double(dfl x) { return (double)x.h + (double)x.l; }

// 1/x: the FP32 reciprocal y and one Newton step y + y (1 - x y), with 1 - x y
// formed exactly to first order (relative error about 2^-47).
DFI dfl df_rcp(dfl x) {
    const float y = f_rcp(x.h);
    const dfl p = df_mul_f(x, y);                      // x y = 1 - r
    const float r = f_sub(f_sub(1.0f, p.h), p.l);      // 1 - p.h is exact
    return fast_two_sum_f(y, f_mul(y, r));
}
// sqrt(x), x >= 0: the FP32 root y and one Newton step y + (x - y^2) / (2y).
DFI dfl df_sqrt(dfl x) {
    if (!(x.h > 0.0f)) return dfl{0.0f, 0.0f};
    const float y = f_sqrt(x.h);
    const float p = f_mul(y, y);
    const float pe = f_fma(y, y, -p);
    const float r = f_add(f_sub(f_sub(x.h, p), pe), x.l);   // x.h - p is exact
    return fast_two_sum_f(y, f_mul(r, f_mul(0.5f, f_rcp(y))));
}

// A double in [2^-74, 2^127] (or 0, or anything below 2^-74, returned as 0)
// as a double-float, from its bits alone: the top 24 significant bits as h,
// the other 29 as l (rounded to 24), renormalised. No FP64 instruction.
DFI dfl df_from_bits(uint32_t hi, uint32_t lo) {
    const uint32_t sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ff);
    if (e < 949) return dfl{0.0f, 0.0f};
    const float h = i_as_f((int32_t)(sgn | ((uint32_t)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29)));
    float l = f_mul((float)(lo & 0x1fffffffu), i_as_f((e - 948) << 23));   // 2^(e - 1075)
    if (sgn) l = -l;
    return fast_two_sum_f(h, l);
}
#if defined(__CUDA_ARCH__)
DFI dfl df_from_double(double x) {
    return df_from_bits((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x));
}
#else
DFI dfl df_from_double(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return df_from_bits((uint32_t)(b >> 32), (uint32_t)b);
}
#endif

// ------------------------------------------------------- exp and log (tables)
// exp(x) for x in [-80, 80] with a normal result: x = (64 m + j) ln2/64 + r,
// |r| <= ln2/128 (+ rounding), ln2/64 in three parts (the first of 9 bits, so
// k times it is exact for |k| < 2^15); e^r = 1 + r + r^2/2 + r^3 (1/6 + r/24 +
// r^2/120) with r^2/2 in double-float (truncation below 4e-17); then 2^(j/64)
// from the table and 2^m by scaling. Relative error about 2^-46.
DFD dfl df_exp(dfl x) {
    const float kf = f_rint(f_mul(x.h, 92.332482616893658f));          // 64 / ln 2
    const int k = (int)kf;
    // ln2/64 = C1 + C2 + C3
    const float C1 = 0x1.63p-7f;                                       // 9 bits
    const float C2 = (float)(0.010830424696249145 - (double)0x1.63p-7f);
    const float C3 = (float)(0.010830424696249145 - (double)0x1.63p-7f - (double)C2);
    const float t = f_fma(-kf, C1, x.h);                               // exact
    const float p2 = f_mul(kf, C2), p2e = f_fma(kf, C2, -p2);
    const dfl s = two_sum_f(t, -p2);
    const dfl r = two_sum_f(s.h, f_add(s.l, f_sub(f_sub(x.l, p2e), f_mul(kf, C3))));
    const dfl r2h = df_scale(df_sqr(r), 0.5f);
    const float rh = r.h;
    const float q = f_fma(f_fma(rh, 1.0f / 120.0f, 1.0f / 24.0f), rh, 1.0f / 6.0f);
    const float tail = f_mul(f_mul(f_mul(rh, rh), rh), q);
    const dfl p = df_add_f(df_add(r, r2h), tail);                       // e^r - 1
    const int j = k & 63, m = k >> 6;
#if defined(__CUDA_ARCH__)
    const dfl T = dfl{__ldg(EXPF_T_HI + j), __ldg(EXPF_T_LO + j)};
#else
    const dfl T = dfl{EXPF_T_HI[j], EXPF_T_LO[j]};
#endif
    const dfl res = df_add(T, df_mul(T, p));
    return df_scale(res, i_as_f((m + 127) << 23));
}

// ln x for x a positive normal double-float: x = 2^e (mh + ml), mh in [1, 2),
// c the table's float nearest 1/(1 + (j + 1/2)/128) for the top 7 fraction bits
// j of mh, r = (mh + ml) c - 1 exactly to first order (|r| < 2^-7.9), ln(1 + r) =
// r - r^2/2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6) with r - r^2/2 in double-float
// (truncation below 3e-18), plus -ln c (table) and e ln 2. Absolute error about
// 2^-47 max(1, |ln x|).
DFD dfl df_log(dfl x) {
    const int32_t b = f_as_i(x.h);
    const int e = ((b >> 23) & 0xff) - 127;
    const int j = (b >> 16) & 127;
    const float mh = i_as_f((b & 0x007fffff) | 0x3f800000);
    const float ml = f_mul(x.l, i_as_f((127 - e) << 23));              // x.l 2^-e
#if defined(__CUDA_ARCH__)
    const float c = __ldg(LOGF_INV_C + j);
    const dfl nl = dfl{__ldg(LOGF_NLN_HI + j), __ldg(LOGF_NLN_LO + j)};
#else
    const float c = LOGF_INV_C[j];
    const dfl nl = dfl{LOGF_NLN_HI[j], LOGF_NLN_LO[j]};
#endif
    const float p = f_mul(mh, c), pe = f_fma(mh, c, -p);
    const dfl r = two_sum_f(f_sub(p, 1.0f), f_fma(ml, c, pe));         // p - 1 is exact
    const float rh = r.h;
    const float q = f_fma(f_fma(f_fma(rh, -1.0f / 6.0f, 0.2f), rh, -0.25f), rh, 1.0f / 3.0f);
    const float tail = f_mul(f_mul(f_mul(rh, rh), rh), q);
    const dfl l1 = df_add_f(df_sub(r, df_scale(df_sqr(r), 0.5f)), tail);
    const dfl eln2 = df_mul_f(DFC(0.6931471805599453094), (float)e);
    return df_add(df_add(eln2, nl), l1);
}

// ------------------------------------------------------------- sin and cos
// sin x and cos x for |x| < 2^7 pi/2: r = x - k pi/2 with pi/2 in three parts
// (the first of 17 bits, so k times it is exact for |k| < 2^7), |r| <= pi/4
// (+ rounding); sin r = r (1 + s(-1/6 + s(1/120 + s(-1/5040 + s(1/9! + s T(s))))))
// and cos r = 1 + s(-1/2 + s(1/24 + s(-1/720 + s(1/8! + s U(s))))), s = r^2, with
// the bracketed steps in double-float and the tails T, U (the Taylor terms from
// s^5/11! and s^5/10! on, to s^7 and s^8) in FP32 (truncation below 1e-16);
// then the quadrant's swap and signs. Absolute error about 1e-15.
DFI void df_sincos(dfl x, dfl &sn, dfl &cs) {
    const float kf = f_rint(f_mul(x.h, 0.63661977236758134f));          // 2 / pi
    const float P1 = 0x1.921fp+0f;                                      // 17 bits
    const float P2 = (float)(1.5707963267948966 - (double)0x1.921fp+0f);
    const float P3 = (float)(1.5707963267948966 - (double)0x1.921fp+0f - (double)P2
                             + 6.123233995736766e-17);
    const float t = f_fma(-kf, P1, x.h);                               // exact
    const float p2 = f_mul(kf, P2), p2e = f_fma(kf, P2, -p2);
    const dfl s0 = two_sum_f(t, -p2);
    const dfl r = two_sum_f(s0.h, f_add(s0.l, f_sub(f_sub(x.l, p2e), f_mul(kf, P3))));
    const dfl s = df_sqr(r);
    const float sh = s.h;
    // tails (Taylor coefficients of sin r / r and cos r from s^5 on)
    const float T = f_fma(f_fma(sh, -1.0f / 1307674368000.0f, 1.0f / 6227020800.0f), sh, -1.0f / 39916800.0f);
    const float U = f_fma(f_fma(f_fma(sh, 1.0f / 20922789888000.0f, -1.0f / 87178291200.0f), sh,
                                1.0f / 479001600.0f), sh, -1.0f / 3628800.0f);
    dfl a = df_add_f(DFC(1.0 / 362880.0), f_mul(sh, T));
    a = df_add(DFC(-1.0 / 5040.0), df_mul(s, a));
    a = df_add(DFC(1.0 / 120.0), df_mul(s, a));
    a = df_add(DFC(-1.0 / 6.0), df_mul(s, a));
    a = df_add_f(df_mul(s, a), 1.0f);
    const dfl sr = df_mul(r, a);
    dfl c = df_add_f(DFC(1.0 / 40320.0), f_mul(sh, U));
    c = df_add(DFC(-1.0 / 720.0), df_mul(s, c));
    c = df_add(DFC(1.0 / 24.0), df_mul(s, c));
    c = df_add_f(df_mul(s, c), -0.5f);
    const dfl cr = df_add_f(df_mul(s, c), 1.0f);
    const int q = ((int)kf) & 3;
    const dfl a0 = (q & 1) ? cr : sr, a1 = (q & 1) ? sr : cr;
    sn = (q & 2) ? df_neg(a0) : a0;
    cs = ((q + 1) & 2) ? df_neg(a1) : a1;
}

}  // namespace gwns
