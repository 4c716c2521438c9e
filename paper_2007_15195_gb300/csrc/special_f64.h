// special_f64.h -- FP64 normal CDF and quantile for the FP64 Genz kernel.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so these forms spend FP64
// operations only where the value needs double precision and do the rest
// (table indices, exponent handling, the quantile's first guess) with
// integer and FP32 instructions:
//
//   Phi(-a), a >= 0:  T = exp(-a^2/2) R(a), R(a) = erfcx(a/sqrt 2)/2 a
//     piecewise degree-8 polynomial (intervals of width 1/8), the exponential
//     table-driven (2^(j/256), two-constant reduction, Taylor to r^4), a^2
//     carried as an exact sum hi + lo; about 23 FP64 operations, relative
//     error ~1e-15 (tables and method: special_f64.cuh, fit_special64.py).
//   Phi^{-1}(s), s = min(p, q): a first guess a0 from the FP32 quantile of
//     the mixed path (evaluated from log2 p + log2 q, taken from the doubles'
//     exponents and mantissas, so it needs no FP64 operation and never
//     underflows), then one Halley step on T(a) = s in FP64:
//         d = (T(a0) - s) / phi(a0),   a1 = a0 + d (1 + a0 d / 2)
//     (phi = -T'(a); the quotient from rcp.approx.f64 and one Newton
//     correction).  The guess is within ~2e-7 relative, so a1 is within
//     ~1e-15 relative (cubic convergence).
//
// The tables live in shared memory (Tables64, filled once per CTA).
#pragma once

#include <stdint.h>

#include "special_f32.h"
#include "special_f64.cuh"

namespace vk {
namespace special64 {

constexpr double kSqrt2PiInv = 0.398942280401432677939946;  // 1 / sqrt(2 pi)
constexpr double kMagic = 6755399441055744.0;                // 1.5 2^52: round to an integer in the low word

struct Tables64 {
    double R[kRIntervals][kRStride];
    double E[1 << kExpBits];
};

// Copy the tables into shared memory (all threads of the CTA; caller syncs).
__device__ __forceinline__ void load_tables(Tables64& t) {
    const double* r = &kR[0][0];
    double* dr = &t.R[0][0];
    for (int i = threadIdx.x; i < kRIntervals * kRStride; i += blockDim.x) dr[i] = r[i];
    for (int i = threadIdx.x; i < (1 << kExpBits); i += blockDim.x) t.E[i] = kExp2Frac[i];
}

__device__ __forceinline__ double rcp_approx(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 2^n as a double for -1022 <= n <= 1023 (integer instructions only).
__device__ __forceinline__ double pow2i(int n) { return __hiloint2double((n + 1023) << 20, 0); }

// Comparisons of non-negative doubles as integers: for x, y >= +0 (and NaN
// above +inf) the bit patterns order as the values, so these take the integer
// pipe instead of GB300's 1/64-rate FP64 pipe.
__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double max_nonneg(double x, double y) {
    return __longlong_as_double(max(bits(x), bits(y)));
}
__device__ __forceinline__ double abs_bits(double x) { return __longlong_as_double(bits(x) & 0x7fffffffffffffffll); }
__device__ __forceinline__ bool sign_bit(double x) { return bits(x) < 0; }

// T = Phi(-a) for a >= 0, and (WANT_PHI) phi(a) = exp(-a^2/2)/sqrt(2 pi).
template <bool WANT_PHI>
__device__ __forceinline__ double tail(const Tables64& tb, double a, double& phi) {
    if (bits(a) >= 0x4043600000000000ll) {  // a >= 38.75 (and inf, NaN): Phi(-a) below the smallest double
        if constexpr (WANT_PHI) phi = 0.0;
        return 0.0;
    }
    // R(a) on the interval whose centre i/8 is nearest to a
    const double ti = fma(a, kRScale, kMagic);
    int i = __double2loint(ti);
    i = min(max(i, 0), kRIntervals - 1);
    const double* c = tb.R[i];
    const double d = a + c[kRDeg + 1];
    double Rv = c[kRDeg];
#pragma unroll
    for (int k = kRDeg - 1; k >= 0; --k) Rv = fma(Rv, d, c[k]);
    // a^2 = hi + lo exactly
    const double hi = a * a;
    const double lo = fma(a, a, -hi);
    // exp(-(hi + lo)/2): k = round(-hi 128/ln2), s = -hi - k ln2/128 - lo = 2 r
    // with |r| <= ln2/512; exp(r) = exp(s/2) by its Taylor polynomial in s
    // (every step scaled by 2, so no halving of a^2 is needed)
    const double tk = fma(-hi, 0.5 * kExpInv, kMagic);
    const int k = __double2loint(tk);
    const double kd = tk - kMagic;
    double r2 = fma(kd, -2.0 * kExpHi, -hi);
    r2 = fma(kd, -2.0 * kExpLo, r2);
    r2 = r2 - lo;
    double p = fma(fma(fma(r2, 1.0 / 384.0, 1.0 / 48.0), r2, 0.125), r2, 0.5);
    p = fma(p, r2, 1.0);
    const double e = tb.E[k & ((1 << kExpBits) - 1)] * p;  // 2^(j/256) exp(r), in [1, 2)
    const int n = k >> kExpBits;                            // -1084 < n <= 0
    const double v = e * Rv;                                // R(a) >= 0.0103: v in [2^-7, 2)
    double T;
    if (n >= -1000) {  // v 2^n stays normal: add n to the exponent field
        T = __hiloint2double(__double2hiint(v) + (n << 20), __double2loint(v));
        if constexpr (WANT_PHI) {
            const double w = e * kSqrt2PiInv;
            phi = __hiloint2double(__double2hiint(w) + (n << 20), __double2loint(w));
        }
    } else {  // near or below the normal range: two exact scalings
        const double s1 = pow2i(-1000), s2 = pow2i(n + 1000);
        T = (v * s1) * s2;
        if constexpr (WANT_PHI) phi = ((e * kSqrt2PiInv) * s1) * s2;
    }
    return T;
}

// Phi(z) and 1 - Phi(z), the smaller one from the tail to full precision.
__device__ __forceinline__ void phi_pair(const Tables64& tb, double z, double& e, double& ec) {
    double unused;
    const double t = tail<false>(tb, abs_bits(z), unused);
    const double u = 1.0 - t;
    const bool neg = sign_bit(z);  // -0 takes the first branch: t = u = 1/2 there
    e = neg ? t : u;
    ec = neg ? u : t;
}

// log2 of a positive normal double as an FP32 value (exponent and the top 20
// mantissa bits: integer instructions and one lg2.approx).
__device__ __forceinline__ float log2_f32(double v) {
    const int hiw = __double2hiint(v);
    const int ex = ((hiw >> 20) & 0x7ff) - 1023;
    const float m = __int_as_float(0x3f800000 | ((hiw & 0xfffff) << 3));  // 1.m
    return (float)ex + special::lg2(m);
}

// A double in [0, 1] as FP32, truncated (values below 2^-126 give 0).
__device__ __forceinline__ float to_f32_unit(double v) {
    const int hiw = __double2hiint(v), low = __double2loint(v);
    const int ex = ((hiw >> 20) & 0x7ff) - 1023 + 127;
    if (ex <= 0) return 0.0f;
    return __int_as_float((ex << 23) | ((hiw & 0xfffff) << 3) | (int)((unsigned)low >> 29));
}

// A non-negative FP32 value as a double (exact; integer instructions).
__device__ __forceinline__ double to_f64_pos(float f) {
    const int b = __float_as_int(f);
    const int ex = (b >> 23) & 0xff;
    if (ex == 0) return 0.0;
    return __hiloint2double(((ex - 127 + 1023) << 20) | ((b & 0x7fffff) >> 3), (b & 7) << 29);
}

// Phi^{-1}(p) given p and q = 1 - p: from the smaller of the two, clamped at
// 2^-1000 (as the definition's quantile).
__device__ __forceinline__ double phiinv_pq(const Tables64& tb, double p, double q) {
    const double lo = 9.3326361850321887899e-302;  // 2^-1000
    const double pc = max_nonneg(p, lo), qc = max_nonneg(q, lo);  // p, q >= 0
    const bool lower = bits(pc) <= bits(qc);
    const double s = lower ? pc : qc;
    const double o = lower ? qc : pc;
    // first guess: the FP32 quantile's magnitude from L = log2(s o)
    const float L = log2_f32(s) + log2_f32(o);
    float f;
    if (L > special::kINV1Lmin)
        f = special::horner(special::kINV1C, fmaf(L, special::kINV1LA, special::kINV1LB));
    else
        f = special::finv_tail(__fmul_rn(-special::kLn2, __fadd_rn(L, 2.0f)));
    const float a0f = fmaxf(__fmul_rn(__fsub_rn(to_f32_unit(o), to_f32_unit(s)), f), 0.0f);
    const double a0 = to_f64_pos(a0f);
    const double ha0 = to_f64_pos(__fmul_rn(a0f, 0.5f));  // a0 / 2 exactly
    // one Halley step on T(a) = s
    double phi;
    const double T = tail<true>(tb, a0, phi);
    const double num = T - s;
    const double rinv = rcp_approx(phi);
    double d = num * rinv;
    d = fma(fma(-phi, d, num), rinv, d);
    const double a1 = fma(d, fma(ha0, d, 1.0), a0);
    return __longlong_as_double(bits(a1) ^ (lower ? (long long)0x8000000000000000ull : 0ll));  // -a1 below 1/2
}

}  // namespace special64
}  // namespace vk
