// special_f32.h -- FP32 normal CDF and quantile for the mixed Genz kernel,
// with a log-space path for probabilities below 2^-64.
//
// Phi of the lower tail (Numerical Recipes "erfcc" form, own coefficients):
//     Phi(-z) = t 2^(a),  t = 1/(1 + z/(2 sqrt 2)),  a = -z^2 log2(e)/2 + P(t),  z >= 0.
// log2 Phi(-z) = log2 t + a is available without underflow.
// Phi^{-1} (M. Giles' erfinv form, own coefficients), from p and q = 1 - p:
//     Phi^{-1}(p) = (p - q) f_s(w),  w = -ln(4 p q),  f_s = sqrt(2) erfinv(y)/y,
// the sign coming from p - q; the central piece is evaluated straight from
// L = log2(p q).  From a log-probability (r < 2^-64): w = -(ln 4 + ln r).
// Coefficients: special_f32.cuh (generated by fit_special.py).  Products and
// sums are written with explicit rounding (__fmul_rn, __fsub_rn, fmaf) so the
// compiler cannot contract them differently from one instantiation to the
// next: every kernel variant computes bit-identical values.
#pragma once

#include "special_f32.cuh"

namespace vk {
namespace special {

constexpr float kLn2 = 0.693147180559945309f;
constexpr float kLn4 = 1.38629436111989062f;
constexpr float kSqrt2 = 1.41421356237309505f;
constexpr float kTinyZ = -9.0f;   // Phi(-9) ~ 2^-62.5: below, carry log2 Phi instead

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Polynomial sum_k c_k u^k by Horner's rule (measured faster here than
// Estrin's scheme, which VK_ESTRIN selects: pairs c_k + c_{k+1} u combined by
// u^2, u^4, u^8 -- a shorter dependent chain for a few more instructions and
// registers).
template <int N>
__device__ __forceinline__ float horner(const float (&c)[N], float u) {
#ifndef VK_ESTRIN
    float acc = c[N - 1];
#pragma unroll
    for (int k = N - 2; k >= 0; --k) acc = fmaf(acc, u, c[k]);
    return acc;
#else
    constexpr int M = (N + 1) / 2;  // pairs
    float a[M];
#pragma unroll
    for (int k = 0; k < M; ++k) a[k] = (2 * k + 1 < N) ? fmaf(c[2 * k + 1], u, c[2 * k]) : c[2 * k];
    float x = __fmul_rn(u, u);
    int m = M;
#pragma unroll
    for (int level = 0; level < 4; ++level) {
        if (m <= 1) break;
        const int h = (m + 1) / 2;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < h) a[k] = (2 * k + 1 < m) ? fmaf(a[2 * k + 1], x, a[2 * k]) : a[2 * k];
        m = h;
        if (m > 1) x = __fmul_rn(x, x);
    }
    return a[0];
#endif
}

// Phi(z) and 1 - Phi(z); for z < kTinyZ also log2 Phi(z) (then e may be 0).
__device__ __forceinline__ void phi_pair(float z, float& e, float& ec, bool& tiny, float& le2) {
    const float az = fminf(fabsf(z), kZmax);
    const float t = rcp(fmaf(az, kKt, 1.0f));
    const float a = fmaf(__fmul_rn(az, -0.5f * kLog2e), az, horner(kPHIC, t));
    const float tail = __fmul_rn(t, ex2(a));  // Phi(-|z|)
    const bool neg = z < 0.0f;
    e = neg ? tail : __fsub_rn(1.0f, tail);
    ec = neg ? __fsub_rn(1.0f, tail) : tail;
    tiny = z < kTinyZ;
    if (tiny) le2 = lg2(t) + a;
}

// Phi(z) and 1 - Phi(z) without the log-space output (e flushes to 0 below
// 2^-126; beyond the fitted |z| <= 38 the exponent only grows more negative).
__device__ __forceinline__ void phi_pair_fast(float z, float& e, float& ec) {
    const float az = fabsf(z);
    const float t = rcp(fmaf(az, kKt, 1.0f));
    const float a = fmaf(__fmul_rn(az, -0.5f * kLog2e), az, horner(kPHIC, t));
    const float tail = __fmul_rn(t, ex2(a));
    const bool neg = z < 0.0f;
    e = neg ? tail : __fsub_rn(1.0f, tail);
    ec = neg ? __fsub_rn(1.0f, tail) : tail;
}

// The same Phi for the mixed Genz step, whose recursion tables carry the
// factor kZs = sqrt(log2(e)/2) (folded into each row's FP64 scaling): from
// zs = kZs z the exponent -z^2 log2(e)/2 is the single fma -zs zs + P(t), and
// t = 1/(1 + z kKt) = 1/(1 + zs kKtS).  Same t and exponent as phi_pair and
// phi_pair_fast up to the FP32 rounding of zs.
constexpr double kZsD = 0.84932180028801904272;  // sqrt(log2(e) / 2)
constexpr float kZs = (float)kZsD;
constexpr float kKtS = (float)(0.35355339059327376220 / kZsD);   // 1 / (2 sqrt(2) kZs)
constexpr float kZmaxS = (float)(38.0 * kZsD);
constexpr float kTinyZS = (float)(-9.0 * kZsD);

__device__ __forceinline__ void phi_pair_s(float zs, float& e, float& ec, bool& tiny, float& le2) {
    const float az = fminf(fabsf(zs), kZmaxS);
    const float t = rcp(fmaf(az, kKtS, 1.0f));
    const float a = fmaf(-az, az, horner(kPHIC, t));
    const float tail = __fmul_rn(t, ex2(a));
    const bool neg = zs < 0.0f;
    e = neg ? tail : __fsub_rn(1.0f, tail);
    ec = neg ? __fsub_rn(1.0f, tail) : tail;
    tiny = zs < kTinyZS;
    if (tiny) le2 = lg2(t) + a;
}

__device__ __forceinline__ void phi_pair_fast_s(float zs, float& e, float& ec) {
    const float az = fabsf(zs);
    const float t = rcp(fmaf(az, kKtS, 1.0f));
    const float a = fmaf(-az, az, horner(kPHIC, t));
    const float tail = __fmul_rn(t, ex2(a));
    const bool neg = zs < 0.0f;
    e = neg ? tail : __fsub_rn(1.0f, tail);
    ec = neg ? __fsub_rn(1.0f, tail) : tail;
}

// f_s(w) = sqrt(2) erfinv(y)/y for w >= 8 (sqrt(w) pieces).
__device__ __forceinline__ float finv_tail(float w) {
    const float s = sqrt_approx(w);  // w = +inf gives s = +inf: the last piece at its end
    if (s < 6.0f) return horner(kINV2C, fmaf(s, kINV2A, kINV2B));  // w in [8, 36)
    if (s < 11.4017543f) return horner(kINV3C, fmaf(s, kINV3A, kINV3B));
    return horner(kINV4C, fmaf(fminf(s, 26.4575131f), kINV4A, kINV4B));
}

// Phi^{-1}(p) given p and q = 1 - p (both >= 0).  w depends on p q only and
// the sign on p - q, so no min/max is needed; p q = 0 (or below the normal
// range) gives L = -inf and the far-tail piece at its end, a finite value.
// Every lane evaluates the central piece; the tail pieces (p q < 2^-13.5,
// rarely reached) run only when a warp vote says some lane needs them.
__device__ __forceinline__ float phiinv_pq(float p, float q) {
    const float L = lg2(__fmul_rn(p, q));  // w = -ln 2 (L + 2)
    float f = horner(kINV1C, fmaf(L, kINV1LA, kINV1LB));
    const bool tail = !(L > kINV1Lmin);
    if (__any_sync(__activemask(), tail)) {  // among the lanes executing this call
        const float ft = finv_tail(__fmul_rn(-kLn2, __fadd_rn(L, 2.0f)));
        f = tail ? ft : f;
    }
    return __fmul_rn(__fsub_rn(p, q), f);
}

// The same quantile in three parts for callers that vote once for several
// values: the central factor f (and whether the tail pieces are needed), the
// tail factor where needed, and (p - q) f.  Same arithmetic as phiinv_pq.
__device__ __forceinline__ float phiinv_central(float p, float q, bool& tail) {
    const float L = lg2(__fmul_rn(p, q));
    tail = !(L > kINV1Lmin);
    return horner(kINV1C, fmaf(L, kINV1LA, kINV1LB));
}
__device__ __forceinline__ float phiinv_with_tail(float p, float q, bool tail, float f) {
    const float L = lg2(__fmul_rn(p, q));
    const float ft = finv_tail(__fmul_rn(-kLn2, __fadd_rn(L, 2.0f)));
    return tail ? ft : f;
}
__device__ __forceinline__ float phiinv_finish(float p, float q, float f) {
    return __fmul_rn(__fsub_rn(p, q), f);
}

// Phi^{-1}(p) from pk = 16 p and qk = 16 q, as the mixed Genz step carries
// them (16 w = |int32(X)| 2^-27 is as exact as w, and so are 16 w e and
// 16 (1 - w e)): L' = log2(pk qk) = log2(p q) + 8 is the central polynomial's
// variable as it stands (kINV1SC: fitted on w = -ln 2 (L' - 6) in
// [0, 12 ln 2], where the map to [-1, 1] is -L'/6 with no offset, folded into
// the coefficients with the factor 1/16), so that Phi^{-1}(p) = (pk - qk) f.
// Split as phiinv_central / phiinv_with_tail for one vote over several values.
__device__ __forceinline__ float phiinv16_central(float pk, float qk, bool& tail) {
    const float L = lg2(__fmul_rn(pk, qk));
    tail = !(L > kINV1SLmin);
    return horner(kINV1SC, L);
}
__device__ __forceinline__ float phiinv16_with_tail(float pk, float qk, bool tail, float f) {
    const float L = lg2(__fmul_rn(pk, qk));
    const float ft = __fmul_rn(finv_tail(fmaf(-kLn2, L, 6.0f * kLn2)), 0.0625f);
    return tail ? ft : f;
}
__device__ __forceinline__ float phiinv16_pq(float pk, float qk) {
    bool tail;
    float f = phiinv16_central(pk, qk, tail);
    if (__any_sync(__activemask(), tail)) f = phiinv16_with_tail(pk, qk, tail, f);
    return __fmul_rn(__fsub_rn(pk, qk), f);
}

// Phi^{-1}(r) for r = 2^lr2 < 2^-64 (log2 input).
__device__ __forceinline__ float phiinv_log2(float lr2) {
    const float w = -fmaf(kLn2, fmaxf(lr2, -1009.0f), kLn4);
    return -finv_tail(w);
}

}  // namespace special
}  // namespace vk
