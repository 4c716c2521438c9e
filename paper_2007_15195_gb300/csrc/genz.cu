// genz.cu -- the fused per-term kernel of the Vecchia log-CDF and the log-sum.
//
// One CTA takes one Vecchia term at a time (a site i of a problem):
//   prologue (one warp, FP64): the block b = (N_i ascending, i) of
//     Sec. 2.2 / Eq. (vecchia-cdf), its covariance from the covariance
//     function (Sec. 3, Sec. 4.1), the Cholesky factor with lanes over rows;
//   body (all warps): Genz's separation-of-variables recursion at the
//     shifted lattice points, one lane per point, the numerator (d-dim) and
//     denominator ((d-1)-dim, the leading block) sharing every sample;
//   epilogue: per-shift lattice means num[i,s], den[i,s] in FP64.
// The log-sum kernel then forms each term on the log scale and sums them in a
// fixed order (Sec. 3.1), with the delta-method standard error over shifts.
//
// Genz's recursion for the d-dim CDF at u with Cholesky factor L (variables
// v = 0..d-1, lattice coordinates t = 0..d-2):
//   e_0 = Phi(u_0 / L_00)
//   y_t = Phi^{-1}(w_t e_t),  w_t = tent(x_t) = 1 - |2 x_t - 1|
//   e_{t+1} = Phi((u_{t+1} - sum_{j<=t} L_{t+1,j} y_j) / L_{t+1,t+1})
//   numerator sample = e_0 ... e_{d-1},  denominator sample = e_0 ... e_{d-2}.
// The partial sums u_v - sum_j L_vj y_j of all later variables are kept in
// registers and updated right after each y_t (right-looking), so the loop over
// t runs at run time with a fixed register array per lane.
//
// A term is a block of d variables whose first c are the conditioning set:
// one site i with c = |N_i| (Eq. vecchia-cdf), or a group of p sites with
// its conditioning set (Sec. 3.2).  Its denominator is the c-dim CDF of the
// leading block, i.e. the product e_0 ... e_{c-1} of the same run (1 when
// c = 0); the numerator is the full product.
#include <cfloat>
#include <climits>
#include <map>
#include <mutex>
#include <tuple>

#include "cov.cuh"
#include "special_f32.h"
#include "special_f64.h"
#include "vk_internal.h"

namespace vk {
namespace {

constexpr int kMaxWarps = 16;
constexpr int kMaxUnits = 64;  // shifts x slices handled by one CTA item

// Entry e of a packed lower triangle (row-major: e = r (r + 1) / 2 + c, c <= r).
__device__ __forceinline__ void tri_index(int e, int& r, int& c) {
    r = (int)((sqrtf((float)(8 * e + 1)) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    while (r * (r + 1) / 2 > e) --r;
    c = e - r * (r + 1) / 2;
}

// Shared memory of a CTA: this fixed part, then (mixed path) the dynamic
// tail dfix[S][DMAX] (the shifts in 32-bit fixed point) and
// stepw[warps][DMAX] (per warp, the step constants of its current shift).
template <int DMAX, bool MIXED>
struct GenzSmem {
    using T = typename std::conditional<MIXED, float, double>::type;
    double A[DMAX][DMAX + 1];  // covariance block, overwritten by its Cholesky factor
    double bx[DMAX], by[DMAX], bu[DMAX];
    double diag[DMAX];
    int bidx[DMAX];            // the block's ordered sites
    // Recursion tables, step t (lattice coordinate t, variable t + 1 next):
    //   Lz[t]      = L_{t+1,t}          coefficient of y_t in variable t+1
    //   Lup[t][r]  = L_{t+2+r,t}        coefficients of y_t in the later variables
    // MIXED multiplies each row v by kZs/L_vv (so the conditional mean arrives
    // standardised and times kZs = sqrt(log2(e)/2), the form its Phi takes);
    // FP64 keeps them unscaled and multiplies the conditional mean by 1/L_vv
    // (diag), one rounding more than the definition's division.
    static constexpr int LS = (DMAX + 3) & ~3;  // row stride: 16-byte aligned rows
    __align__(16) T Lup[DMAX][LS];
    __align__(16) T Lz[DMAX];
    __align__(16) T up[DMAX];  // MIXED: kZs u_v / L_vv;  FP64: u_v
    uint32_t gl[DMAX];         // FP64: g_t;  MIXED: round(g_t 2^32 / N)
    uint64_t g64[MIXED ? 1 : DMAX];  // FP64: round(g_t 2^64 / N)
    double part_num[kMaxUnits], part_den[kMaxUnits];
    double e0, ec0;
    float le2_0;  // log2 e0 when e0 < 2^-64 (mixed path)
    int q, c, bad, flag;
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// FP64 path, per warp and step of its current shift: the lattice coordinate's
// multiplier and shift in 64-bit fixed point (round(g_t 2^64 / N), Delta_t 2^64)
// and the step's coefficient -L_{t+1,t} and 1/L_{t+1,t+1}.
struct Step64 {
    uint64_t G, D;
    double nlz, rdiag;
};

// Bytes of shared memory for a CTA of `warps` warps on problems with <= max_S
// shifts: the fixed part, then (mixed) the shifts in fixed point and the
// per-warp step constants, or (FP64) the tail tables and the per-warp steps.
template <int DMAX, bool MIXED>
constexpr size_t smem_bytes(int max_S, int warps) {
    return align16(sizeof(GenzSmem<DMAX, MIXED>)) +
           (MIXED ? align16((size_t)max_S * DMAX * 4) + (size_t)warps * DMAX * 16
                  : align16(sizeof(special64::Tables64)) + (size_t)warps * DMAX * sizeof(Step64));
}

extern __shared__ __align__(16) unsigned char vk_smem[];

// The dynamic tail: dfix row of shift s, and the step constants of a warp:
// {-L_{t+1,t}/L_{t+1,t+1}, round(g_t 2^32/N), shift_t 2^32, 0}, one 16-byte load per step.
template <int DMAX>
__device__ __forceinline__ uint32_t* dfix_row(int s) {
    return (uint32_t*)(vk_smem + align16(sizeof(GenzSmem<DMAX, true>))) + s * DMAX;
}
template <int DMAX>
__device__ __forceinline__ float4* stepw_of(int max_S, int warp) {
    return (float4*)(vk_smem + align16(sizeof(GenzSmem<DMAX, true>)) + align16((size_t)max_S * DMAX * 4)) +
           warp * DMAX;
}
template <int DMAX>
__device__ __forceinline__ special64::Tables64& tables64() {
    return *reinterpret_cast<special64::Tables64*>(vk_smem + align16(sizeof(GenzSmem<DMAX, false>)));
}
template <int DMAX>
__device__ __forceinline__ Step64* step64_of(int warp) {
    return reinterpret_cast<Step64*>(vk_smem + align16(sizeof(GenzSmem<DMAX, false>)) +
                                     align16(sizeof(special64::Tables64))) +
           warp * DMAX;
}

// Phi(z) and 1 - Phi(z), the smaller one from the tail to full precision.
__device__ __forceinline__ void phi_pair64(double z, double& e, double& ec) {
    const double t = normcdf(-fabs(z));
    e = (z < 0.0) ? t : 1.0 - t;
    ec = (z < 0.0) ? 1.0 - t : t;
}


// 2^-E as a double (0 once below the normal range).
__device__ __forceinline__ double pow2_neg(int E) {
    return (E < 1022) ? __longlong_as_double((long long)(1023 - E) << 52) : 0.0;
}

// ------------------------ mixed (FP32 integrand) path ------------------------
// Per lane and point: the standardised partial sums R of the later variables,
// the current conditional probability e (and 1 - e, and log2 e once e is below
// 2^-64), and the running product g 2^-E of e_1 .. e_t (e_0 is factored out
// and applied in FP64), its exponent tracked so it never underflows.

template <int DMAX, int P>
struct MixedLanes {
    float R[P][DMAX - 1];
    float e[P], ec[P], le2[P], g[P];
    int E[P];
    bool tiny[P];
    uint32_t kk[P];
};

__device__ __forceinline__ void scale_by(float& g, int& E, float v) {
    g *= v;
    if (g < 0x1p-32f) {
        g *= 0x1p32f;
        E += 32;
    }
}

// g 2^-E times 2^l2 (l2 << 0), kept normal
__device__ __forceinline__ void scale_by_log2(float& g, int& E, float l2) {
    const float k = floorf(l2);
    g *= special::ex2(l2 - k);
    E -= (int)k;
    if (g < 0x1p-32f) {
        g *= 0x1p32f;
        E += 32;
    }
}

// Steps t0 <= t < t1 with update width W: each step needs q - t - 1 <= W.
template <int DMAX, int P, int W>
__device__ __forceinline__ void mixed_steps(const GenzSmem<DMAX, true>& sm, const uint32_t* dfs,
                                            int t0, int t1, MixedLanes<DMAX, P>& L) {
    for (int t = t0; t < t1; ++t) {
        const float* lup = sm.Lup[t];
        const float lz = sm.Lz[t];
        const uint32_t G = sm.gl[t], Dt = dfs[t];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (t > 0) {  // g *= e_t
                if (!L.tiny[p])
                    scale_by(L.g[p], L.E[p], L.e[p]);
                else
                    scale_by_log2(L.g[p], L.E[p], L.le2[p]);
            }
            // lattice coordinate in 32-bit fixed point, tent transform w = 1 - |2x - 1|
            // of x = X 2^-32: exactly |int32(X)| 2^-31
            const uint32_t X = L.kk[p] * G + Dt;
            const uint32_t V = ((int32_t)X < 0) ? 0u - X : X;
            const float w = __uint2float_rn(V) * 0x1p-31f;
            float y;
            if (!L.tiny[p]) {
                const float a = __uint2float_rn(0x80000000u - V) * 0x1p-31f;  // |2x - 1|
                y = special::phiinv_pq(w * L.e[p], fmaf(w, L.ec[p], a));
            } else {  // w e_t below 2^-64: from log2(w e_t)
                y = special::phiinv_log2(special::lg2(w) + L.le2[p]);
            }
            const float z = fmaf(-lz, y, L.R[p][0]);  // kZs z (the tables carry kZs)
#pragma unroll
            for (int r = 0; r < W; ++r) L.R[p][r] = fmaf(-lup[r], y, L.R[p][r + 1]);
            special::phi_pair_s(z, L.e[p], L.ec[p], L.tiny[p], L.le2[p]);
        }
    }
}

// Steps t <= t' < t_stop of a term with q steps, in phases of update width
// W, W - 8, ...: a step needs width q - t' - 1.
template <int DMAX, int P, int W>
__device__ __forceinline__ void mixed_phases(const GenzSmem<DMAX, true>& sm, const uint32_t* dfs,
                                             int t, int t_stop, int q, MixedLanes<DMAX, P>& L) {
    constexpr int WN = W - 8;
    const int t_end = (WN > 0) ? max(t, min(t_stop, q - 1 - WN)) : t_stop;
    mixed_steps<DMAX, P, W>(sm, dfs, t, t_end, L);
    if constexpr (WN > 0) mixed_phases<DMAX, P, WN>(sm, dfs, t_end, t_stop, q, L);
}

template <int DMAX, int P>
__device__ __forceinline__ void genz_points_safe(const GenzSmem<DMAX, true>& sm, int q, int c, int s,
                                                  int64_t k_begin, int64_t k_end, double& acc_num,
                                                  double& acc_den) {
    constexpr int W0 = (DMAX - 2 > 0) ? DMAX - 2 : 1;
    const int lane = threadIdx.x & 31;
    const uint32_t* dfs = dfix_row<DMAX>(s);
    const int cut = (c >= 1) ? c : q;  // after steps 0 .. cut-1, g = e_1 ... e_{c-1}
    const float e0f = (float)sm.e0, ec0f = (float)sm.ec0;
    const bool tiny0 = sm.e0 < 0x1p-64;
    for (int64_t kb = k_begin; kb < k_end; kb += 32 * P) {
        MixedLanes<DMAX, P> L;
        bool valid[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int64_t k = kb + p * 32 + lane;
            valid[p] = k < k_end;
            L.kk[p] = (uint32_t)(valid[p] ? k : k_begin);
#pragma unroll
            for (int r = 0; r < DMAX - 1; ++r) L.R[p][r] = sm.up[1 + r];
            L.e[p] = e0f;
            L.ec[p] = ec0f;
            L.tiny[p] = tiny0;
            L.le2[p] = sm.le2_0;
            L.g[p] = 1.0f;
            L.E[p] = 0;
        }
        mixed_phases<DMAX, P, W0>(sm, dfs, 0, cut, q, L);
        double den_c[P];
#pragma unroll
        for (int p = 0; p < P; ++p) den_c[p] = (double)L.g[p] * pow2_neg(L.E[p]);
        mixed_phases<DMAX, P, W0>(sm, dfs, cut, q, q, L);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (valid[p]) {
                const double den = den_c[p];
                float gn = L.g[p];
                int En = L.E[p];
                if (!L.tiny[p])
                    scale_by(gn, En, L.e[p]);
                else
                    scale_by_log2(gn, En, L.le2[p]);
                acc_den += den;
                acc_num += (double)gn * pow2_neg(En);
            }
        }
    }
}

// ------------------- mixed path, fast form (the common case) -----------------
// No log-space bookkeeping: a conditional probability below the FP32 range
// simply zeroes its point's sample.  Such a sample is below 2^-62 in absolute
// terms, so whenever the term's lattice means are at least 2^-40 the loss is
// below 2^-22 relative; terms whose means fall under 2^-40 are flagged and
// re-evaluated by the log-space form above (genz_points_safe).  Sums run in
// FP32 with Kahan compensation per lane and are folded into FP64 per unit.

struct Kahan32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int DMAX, int P, int W, bool FIRST>
__device__ __forceinline__ void fast_step(const GenzSmem<DMAX, true>& sm, const float4* sc, int t,
                                          float (&R)[P][DMAX - 1], float (&e)[P], float (&ec)[P],
                                          float (&g)[P], const uint32_t (&kk)[P]) {
    const float* lup = sm.Lup[t];
    const float4 c = sc[t];
    const float nlz = c.x;  // -L_{t+1,t}/L_{t+1,t+1}
    const uint32_t G = __float_as_uint(c.y), Dt = __float_as_uint(c.z);
    if constexpr (P == 1) {  // one point per lane: the per-point form keeps fewer values live
        if (!FIRST) g[0] = __fmul_rn(g[0], e[0]);
        const uint32_t X = kk[0] * G + Dt;
        const float wk = __fmul_rn(fabsf(__int2float_rn((int32_t)X)), 0x1p-27f);  // 16 w
        const float yv = special::phiinv16_pq(__fmul_rn(wk, e[0]), fmaf(wk, ec[0], __fsub_rn(16.0f, wk)));
        const float z = fmaf(nlz, yv, R[0][0]);
#pragma unroll
        for (int r = 0; r < W; ++r) R[0][r] = fmaf(-lup[r], yv, R[0][r + 1]);
        special::phi_pair_fast_s(z, e[0], ec[0]);
        return;
    }
    // Phi^{-1} of every point's w_t e_t first, so one full-warp vote decides
    // the tail pieces for all of them (every lane of the warp runs this step)
    float pp[P], qq[P], y[P];
    bool tail[P];
    bool any_tail = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!FIRST) g[p] = __fmul_rn(g[p], e[p]);  // g = e_1 ... e_t
        // lattice coordinate in 32-bit fixed point, tent transform w = 1 - |2x - 1|
        // of x = X 2^-32: exactly |int32(X)| 2^-31 (the sign folds into the
        // product); carried as 16 w, 16 w e and 16 (1 - w e), exact scalings
        // that give the quantile's polynomial its variable directly
        const uint32_t X = kk[p] * G + Dt;
        const float wk = __fmul_rn(fabsf(__int2float_rn((int32_t)X)), 0x1p-27f);
        pp[p] = __fmul_rn(wk, e[p]);
        qq[p] = fmaf(wk, ec[p], __fsub_rn(16.0f, wk));
        y[p] = special::phiinv16_central(pp[p], qq[p], tail[p]);
        any_tail = any_tail || tail[p];
    }
    if (__any_sync(0xffffffffu, any_tail)) {
#pragma unroll
        for (int p = 0; p < P; ++p) y[p] = special::phiinv16_with_tail(pp[p], qq[p], tail[p], y[p]);
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float yv = special::phiinv_finish(pp[p], qq[p], y[p]);
        const float z = fmaf(nlz, yv, R[p][0]);  // kZs z (the tables carry kZs)
#pragma unroll
        for (int r = 0; r < W; ++r) R[p][r] = fmaf(-lup[r], yv, R[p][r + 1]);
        special::phi_pair_fast_s(z, e[p], ec[p]);
    }
}

// Width step between phases: 4 up to 21 variables; 6 above, where fewer
// copies of the step body (instruction cache) beat the extra padding FMAs
// (measured: m = 30 5.7 % faster, m <= 16 0.7 % slower with 6).
#ifndef VK_PHASE_STEP_SMALL
#define VK_PHASE_STEP_SMALL 4
#endif
__host__ __device__ constexpr int phase_step(int dmax) { return dmax <= 21 ? VK_PHASE_STEP_SMALL : 6; }

// Steps t <= t' < q (t >= 1) of a term with q steps, in phases of update width
// W, W - step, ...: a step needs width q - t' - 1, so the phase of width W ends
// where W - step suffices.  CAPTURE (terms whose conditioning set is shorter
// than q): at the start of step c (warp-uniform), gd = g = e_1 ... e_{c-1},
// the conditioning CDF's sample.  A classic term (c = q) uses g at the end
// and runs the instantiation without the check.
template <int DMAX, int P, int W, bool CAPTURE>
__device__ __forceinline__ void fast_phases(const GenzSmem<DMAX, true>& sm, const float4* sc, int t,
                                            int q, int cut, float (&R)[P][DMAX - 1], float (&e)[P],
                                            float (&ec)[P], float (&g)[P], float (&gd)[P],
                                            const uint32_t (&kk)[P]) {
    constexpr int WN = W - phase_step(DMAX);
    const int t_end = (WN > 0) ? max(t, min(q, q - 1 - WN)) : q;
    for (int tt = t; tt < t_end; ++tt) {
        if (CAPTURE && tt == cut) {
#pragma unroll
            for (int p = 0; p < P; ++p) gd[p] = g[p];
        }
        fast_step<DMAX, P, W, false>(sm, sc, tt, R, e, ec, g, kk);
    }
    if constexpr (WN > 0) fast_phases<DMAX, P, WN, CAPTURE>(sm, sc, t_end, q, cut, R, e, ec, g, gd, kk);
}

template <int DMAX, int P, bool CAPTURE>
__device__ __forceinline__ void genz_points_fast(const GenzSmem<DMAX, true>& sm, int q, int c, int s,
                                                 int max_S, int64_t k_begin, int64_t k_end,
                                                 double& acc_num, double& acc_den) {
    constexpr int W0 = (DMAX - 2 > 0) ? DMAX - 2 : 1;
    const int lane = threadIdx.x & 31;
    float4* sc = stepw_of<DMAX>(max_S, threadIdx.x >> 5);
    const uint32_t* dfs = dfix_row<DMAX>(s);
    __syncwarp();
    for (int t = lane; t < q; t += 32)
        sc[t] = make_float4(-sm.Lz[t], __uint_as_float(sm.gl[t]), __uint_as_float(dfs[t]), 0.0f);
    __syncwarp();
    const float e0f = (float)sm.e0, ec0f = (float)sm.ec0;
    // point indices in 32 bits: N <= 2^31 - 1, so kb + 32 P stays below 2^32
    const uint32_t k_lo = (uint32_t)k_begin, k_hi = (uint32_t)k_end;
    Kahan32 kn, kd;
    for (uint32_t kb = k_lo; kb < k_hi; kb += 32 * P) {
        float R[P][DMAX - 1], e[P], ec[P], g[P], gd[P];
        uint32_t kk[P];
        bool valid[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const uint32_t k = kb + p * 32 + lane;
            valid[p] = k < k_hi;
            kk[p] = valid[p] ? k : k_lo;
#pragma unroll
            for (int r = 0; r < DMAX - 1; ++r) R[p][r] = sm.up[1 + r];
            e[p] = e0f;
            ec[p] = ec0f;
            g[p] = 1.0f;
            gd[p] = 1.0f;  // c = 1: e_0 alone (factored out)
        }
        fast_step<DMAX, P, W0, true>(sm, sc, 0, R, e, ec, g, kk);  // q >= 1: step 0 at full width
        fast_phases<DMAX, P, W0, CAPTURE>(sm, sc, 1, q, c, R, e, ec, g, gd, kk);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (valid[p]) {
                kd.add(CAPTURE ? gd[p] : g[p]);
                kn.add(__fmul_rn(g[p], e[p]));
            }
        }
    }
    acc_num += kn.value();
    acc_den += kd.value();
}

// ------------------------------- FP64 path ---------------------------------

// Lattice coordinate in 64-bit fixed point to a double: V 2^-63 for
// 0 <= V <= 2^63, rounded to 53 bits (integer instructions only).
__device__ __forceinline__ double fix63_to_f64(uint64_t V) {
    if (V == 0) return 0.0;
    const int lz = __clzll((long long)V);
    const uint64_t m = V << lz;  // bit 63 set
    const uint64_t bits = ((uint64_t)(1023 - lz) << 52) + ((m >> 11) & 0xFFFFFFFFFFFFFull) + ((m >> 10) & 1);
    return __longlong_as_double((long long)bits);
}

// One FP64 step t (lattice coordinate t, variable t + 1 next) of a point:
// update width W.  x = frac(k g_t / N + Delta_t) in 64-bit fixed point
// X = k G_t + D_t mod 2^64; the tent w = 1 - |2x - 1| = |int64(X)| 2^-63
// and |2x - 1| = 1 - w from the same integer.
template <int DMAX, int W>
__device__ __forceinline__ void fp64_step(const GenzSmem<DMAX, false>& sm, const special64::Tables64& tb,
                                          const Step64& st, int t, uint32_t k, double (&R)[DMAX - 1], double& e,
                                          double& ec) {
    const uint64_t X = (uint64_t)k * st.G + st.D;
    const uint64_t V = ((int64_t)X < 0) ? (0ull - X) : X;  // |int64(X)| <= 2^63
    const double w = fix63_to_f64(V);
    const double a = fix63_to_f64((1ull << 63) - V);
    const double pp = w * e;
    const double qq = fma(w, ec, a);
    const double y = special64::phiinv_pq(tb, pp, qq);
    const double* lup = sm.Lup[t];
    const double acc = fma(st.nlz, y, R[0]);
#pragma unroll
    for (int r = 0; r < W; ++r) R[r] = fma(-lup[r], y, R[r + 1]);
    special64::phi_pair(tb, acc * st.rdiag, e, ec);
}

// Steps t <= t' < q in phases of update width W, W - step, ... (as the mixed path).
template <int DMAX, int W>
__device__ __forceinline__ void fp64_phases(const GenzSmem<DMAX, false>& sm, const special64::Tables64& tb,
                                            const Step64* st, int t, int q, int c, uint32_t k,
                                            double (&R)[DMAX - 1], double& e, double& ec, double& f, double& fc) {
    constexpr int WN = W - phase_step(DMAX);
    const int t_end = (WN > 0) ? max(t, min(q, q - 1 - WN)) : q;
    for (int tt = t; tt < t_end; ++tt) {
        f *= e;                   // e_0 ... e_tt
        if (tt + 1 == c) fc = f;  // the c-dim CDF sample of the leading block
        fp64_step<DMAX, W>(sm, tb, st[tt], tt, k, R, e, ec);
    }
    if constexpr (WN > 0) fp64_phases<DMAX, WN>(sm, tb, st, t_end, q, c, k, R, e, ec, f, fc);
}

// 2^64 g / N rounded to the nearest integer (g < N < 2^32), by two steps of
// long division.
__device__ __forceinline__ uint64_t fix64_ratio(uint32_t g, uint64_t N) {
    const uint64_t a = ((uint64_t)g << 32), q1 = a / N, r1 = a % N;
    const uint64_t b = r1 << 32, q2 = b / N, r2 = b % N;
    return (q1 << 32) + q2 + ((2 * r2 >= N) ? 1u : 0u);
}

template <int DMAX>
__device__ __forceinline__ void genz_points_fp64(const GenzSmem<DMAX, false>& sm, const ProbDev& P,
                                                 int q, int c, int s, int64_t k_begin, int64_t k_end,
                                                 double& acc_num, double& acc_den) {
    constexpr int W0 = (DMAX - 2 > 0) ? DMAX - 2 : 1;
    const int lane = threadIdx.x & 31;
    const special64::Tables64& tb = tables64<DMAX>();
    Step64* st = step64_of<DMAX>(threadIdx.x >> 5);
    const double* dl = P.delta + (int64_t)s * P.dim;
    __syncwarp();
    for (int t = lane; t < q; t += 32) {
        // Delta = M 2^-53 exactly (53-bit shifts): D = M 2^11
        const uint64_t M = (uint64_t)__double2ull_rn(dl[t] * 9007199254740992.0);
        st[t] = Step64{sm.g64[t], M << 11, -sm.Lz[t], sm.diag[t + 1]};
    }
    __syncwarp();
    for (int64_t k = k_begin + lane; k < k_end; k += 32) {
        double R[DMAX - 1];
#pragma unroll
        for (int r = 0; r < DMAX - 1; ++r) R[r] = sm.up[1 + r];
        double e = sm.e0, ec = sm.ec0, f = 1.0, fc = 1.0;
        fp64_phases<DMAX, W0>(sm, tb, st, 0, q, c, (uint32_t)k, R, e, ec, f, fc);
        acc_den += fc;
        acc_num += f * e;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Work items: (problem, site, shift group).  A list of segments maps a flat
// item index to them: segment k covers items [seg_prefix[k], seg_prefix[k+1])
// = sites seg_base[k].y, ... of problem seg_base[k].x, each split into
// `groups` shift groups (the group index varies fastest).  With an explicit
// `items` list (the FP64 re-evaluation of flagged sites) an item is
// (problem, site) with all shifts, and its count may live on the device.
//
// The last round of a launch: with items of equal size, a launch of n items
// on a grid of G CTAs leaves n mod G CTAs with one item more than the rest,
// and they finish alone at a fraction of their SMs' throughput.  So the sites
// after `whole_sites` (those whose items would form that last round) are cut
// into `tail_groups` shift groups instead of `groups`: more, smaller items
// that spread over the whole grid.  A shift's partial means are computed by
// one warp whatever the grouping, so the results do not change.
struct ItemSrc {
    const int2* items;       // explicit (problem, site) items, or nullptr
    const int* dev_count;    // device-side count for `items`, or nullptr
    const int* seg_prefix;   // n_segs + 1 prefix sums of items
    const int2* seg_base;    // (problem, first site) per segment
    int n_segs;
    int n_items;
    int groups;              // shift groups per site (segment mode)
    int whole_sites;         // sites [0, whole_sites) in `groups` groups, the rest in tail_groups
    int tail_groups;
    int fb_cap;              // capacity of the flagged-item list
};

__device__ __forceinline__ void item_of(const ItemSrc& src, int it, int2& ps, int& grp, int& ngroups) {
    if (src.items) {
        ps = src.items[it];
        grp = 0;
        ngroups = 1;
        return;
    }
    int site_item;
    const int whole = src.whole_sites * src.groups;
    if (it < whole) {
        site_item = it / src.groups;
        grp = it - site_item * src.groups;
        ngroups = src.groups;
    } else {
        const int j = it - whole, k = j / src.tail_groups;
        site_item = src.whole_sites + k;
        grp = j - k * src.tail_groups;
        ngroups = src.tail_groups;
    }
    int lo = 0, hi = src.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (src.seg_prefix[mid] <= site_item)
            lo = mid;
        else
            hi = mid - 1;
    }
    ps = make_int2(src.seg_base[lo].x, src.seg_base[lo].y + (site_item - src.seg_prefix[lo]));
}

// MODE: 0 = FP64, 1 = mixed fast form, 2 = mixed log-space form.
constexpr int kModeFP64 = 0, kModeFast = 1, kModeSafe = 2;

// Register cap per thread: the fast mixed loop keeps DMAX - 1 partial sums per
// point in registers; capping the rest raises the number of resident warps.
// Blocks above 32 variables run one point per lane with up to 128 registers
// (fast) or 255 (FP64 and log-space forms, whose partial sums are wider), and
// at most 256 threads per CTA.
#ifndef VK_CAP_P1_SMALL
#define VK_CAP_P1_SMALL 64
#endif
#ifndef VK_CAP_P1_LARGE
#define VK_CAP_P1_LARGE 80
#endif
#ifndef VK_CAP_P2_SMALL
#define VK_CAP_P2_SMALL 96
#endif
#ifndef VK_CAP_P2_LARGE
#define VK_CAP_P2_LARGE 128
#endif
__host__ __device__ constexpr int reg_cap(int dmax, int p, int mode) {
    return dmax > 32            ? (mode == kModeFast ? 128 : 255)
           : mode != kModeFast ? 128
           : p == 1            ? (dmax <= 16 ? VK_CAP_P1_SMALL : VK_CAP_P1_LARGE)
                               : (dmax <= 16 ? VK_CAP_P2_SMALL : VK_CAP_P2_LARGE);
}
__host__ __device__ constexpr int max_threads(int dmax, int p, int mode) {
    return reg_cap(dmax, p, mode) > 128 ? 256 : 512;
}

// A term of a problem: its block (the conditioning sites ascending, then the
// sites of the term) into sm.bidx, c and d; false if the row is malformed.
// Classic (group 0): term i is site i with N_i = the first min(m, i) entries
// of row i.  Group p: term k is sites k p .. min(k p + p, D) - 1 with the
// leading non-negative entries of row k (the rest must be -1).
template <int DMAX, bool MIXED>
__device__ __forceinline__ bool term_block(GenzSmem<DMAX, MIXED>& sm, const ProbDev& Pd, int64_t term,
                                           int& c, int& d, int64_t& i0) {
    const int lane = threadIdx.x & 31;
    const int m = Pd.m;
    const int32_t* row = Pd.nbr + term * (int64_t)m;
    int g;
    bool ok = true;
    if (Pd.group == 0) {
        i0 = term;
        g = 1;
        c = (int)((term < m) ? term : m);
    } else {
        i0 = term * Pd.group;
        g = (int)min((int64_t)Pd.group, Pd.D - i0);
        c = m;
        for (int base = 0; base < m; base += 32) {  // first negative entry
            const int r = base + lane;
            const unsigned neg = __ballot_sync(0xffffffffu, r < m && row[r] < 0);
            if (neg) {
                c = base + __ffs(neg) - 1;
                break;
            }
        }
        for (int r = c + lane; r < m; r += 32) ok = ok && row[r] < 0;
    }
    d = c + g;
    if (d > DMAX) ok = false;
    if (ok)
        for (int v = lane; v < d; v += 32) sm.bidx[v] = (v < c) ? row[v] : (int)(i0 + (v - c));
    __syncwarp();
    if (ok)
        for (int v = lane; v < c; v += 32) {
            const int idx = sm.bidx[v];
            ok = ok && idx >= 0 && idx < i0 && (v == 0 || idx > sm.bidx[v - 1]);  // ascending (block order)
        }
    return __all_sync(0xffffffffu, ok);
}

template <int DMAX, int P, int MODE>
__global__ void __launch_bounds__(max_threads(DMAX, P, MODE)) __maxnreg__(reg_cap(DMAX, P, MODE))
    genz_kernel(const ProbDev* __restrict__ probs, ItemSrc src, int slices, int max_S,
                ProbResult* __restrict__ results, int* __restrict__ fallback_count,
                int2* __restrict__ fallback_items) {
    constexpr bool MIXED = MODE != kModeFP64;
    GenzSmem<DMAX, MIXED>& sm = *reinterpret_cast<GenzSmem<DMAX, MIXED>*>(vk_smem);
    using T = typename GenzSmem<DMAX, MIXED>::T;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;

    if constexpr (!MIXED) {
        special64::load_tables(tables64<DMAX>());
        __syncthreads();
    }
    const int n_run = src.dev_count ? min(*src.dev_count, src.n_items) : src.n_items;
    for (int it = blockIdx.x; it < n_run; it += gridDim.x) {
        int2 item;
        int grp, groups;
        item_of(src, it, item, grp, groups);
        const ProbDev& Pd = probs[item.x];
        const int64_t term = item.y;
        const int S = Pd.S;
        const int s_lo = (S * grp) / groups, s_hi = (S * (grp + 1)) / groups;

        // ---- prologue: block (warp 0), covariance (all warps), Cholesky (warp 0); FP64 ----
        if (warp == 0) {
            int c = 0, d = 1;
            int64_t i0 = 0;
            const int bad = term_block<DMAX, MIXED>(sm, Pd, term, c, d, i0) ? 0 : 2;
            if (!bad)
                for (int v = lane; v < d; v += 32) {
                    const int idx = sm.bidx[v];
                    sm.bx[v] = Pd.sites[2 * (int64_t)idx];
                    sm.by[v] = Pd.sites[2 * (int64_t)idx + 1];
                    sm.bu[v] = Pd.u[idx];
                }
            if (lane == 0) {
                sm.bad = bad;
                sm.q = d - 1;
                sm.c = c;
                sm.flag = 0;
            }
        }
        __syncthreads();
        // covariance, lower triangle, entries packed over every thread (the
        // FP64 units of all the CTA's warps)
        if (!sm.bad) {
            const int d = sm.q + 1;
            for (int e = threadIdx.x; e < d * (d + 1) / 2; e += blockDim.x) {
                int r, col;
                tri_index(e, r, col);
                const double h = site_dist(Pd, __dsub_rn(sm.bx[r], sm.bx[col]), __dsub_rn(sm.by[r], sm.by[col]));
                double v = cov_fn(Pd.cov_kind, Pd.variance, Pd.range, Pd.nu, h);
                if (col == r) v += Pd.nugget;
                if (Pd.lr_k > 0) {  // conditional covariance: minus scale V_a . V_b
                    const double* Va = Pd.lr_V + (int64_t)sm.bidx[r] * Pd.lr_k;
                    const double* Vb = Pd.lr_V + (int64_t)sm.bidx[col] * Pd.lr_k;
                    double acc = 0.0;
                    for (int t = 0; t < Pd.lr_k; ++t) acc = fma(Va[t], Vb[t], acc);
                    v = v - Pd.lr_scale * acc;
                }
                sm.A[r][col] = v;
            }
        }
        __syncthreads();
        if (warp == 0 && !sm.bad) {
            const int d = sm.q + 1;
            int bad = 0;
            // Cholesky, right-looking: after column j is final, the trailing
            // triangle takes its update fma(-L_rj, L_cj, A_rc), entries packed
            // over the lanes.  Each entry thus receives its terms in ascending
            // k with fma and is divided by the pivot last: the operations of
            // the row-by-row definition, in its order.
            for (int j = 0; j < d; ++j) {
                const double s = sm.A[j][j];
                if (!(s > 0.0)) {  // warp-uniform: every lane reads the same value
                    bad = 1;
                    break;
                }
                const double piv = sqrt(s);
                for (int r = j + 1 + lane; r < d; r += 32) sm.A[r][j] = sm.A[r][j] / piv;
                __syncwarp();
                if (lane == 0) sm.A[j][j] = piv;
                const int n = d - 1 - j;
                for (int e = lane; e < n * (n + 1) / 2; e += 32) {
                    int a, b;
                    tri_index(e, a, b);
                    const int r = j + 1 + a, col = j + 1 + b;
                    sm.A[r][col] = fma(-sm.A[r][j], sm.A[col][j], sm.A[r][col]);
                }
                __syncwarp();
            }
            if (lane == 0) {
                sm.bad = bad;
                if (!bad) {
                    const double z0 = sm.bu[0] / sm.A[0][0];
                    phi_pair64(z0, sm.e0, sm.ec0);
                    sm.le2_0 = (sm.e0 < 0x1p-64) ? (float)log2(sm.e0) : 0.0f;
                }
            }
        }
        __syncthreads();
        const int q = sm.q, c = sm.c;

        if (!sm.bad) {
            // ---- derived tables for the recursion ----
            // (one FP64 reciprocal 1/L_vv per row; mixed: each row scaled by
            // kZs/L_vv, so the recursion's conditional means arrive as the
            // kZs z that its Phi takes)
            constexpr int LS = GenzSmem<DMAX, MIXED>::LS;
            const int d = q + 1;
            for (int v = threadIdx.x; v < DMAX; v += blockDim.x)
                sm.diag[v] = (v < d) ? (MIXED ? special::kZsD : 1.0) / sm.A[v][v] : 0.0;
            __syncthreads();
            for (int x = threadIdx.x; x < DMAX * LS; x += blockDim.x) {
                const int t = x / LS, r = x % LS, v = t + 2 + r;
                T val = (T)0;
                if (t < q && v < d) {
                    if constexpr (MIXED)
                        val = (T)(sm.A[v][t] * sm.diag[v]);
                    else
                        val = sm.A[v][t];
                }
                sm.Lup[t][r] = val;
            }
            for (int v = threadIdx.x; v < DMAX; v += blockDim.x) {
                T val = (T)0, lz = (T)0;
                if (v < d) {
                    if constexpr (MIXED)
                        val = (T)(sm.bu[v] * sm.diag[v]);
                    else
                        val = sm.bu[v];
                }
                if (v < q) {
                    if constexpr (MIXED)
                        lz = (T)(sm.A[v + 1][v] * sm.diag[v + 1]);
                    else
                        lz = sm.A[v + 1][v];
                }
                sm.up[v] = val;
                sm.Lz[v] = lz;
                if (v < q) sm.gl[v] = MIXED ? Pd.gfix[v] : Pd.g[v];
                if constexpr (!MIXED)
                    if (v < q) sm.g64[v] = fix64_ratio(Pd.g[v], (uint64_t)Pd.N);
            }
            if constexpr (MIXED) {
                for (int x = threadIdx.x; x < S * DMAX; x += blockDim.x) {
                    const int s = x / DMAX, t = x % DMAX;
                    dfix_row<DMAX>(s)[t] = (t < q) ? Pd.dfix[(int64_t)s * Pd.dim + t] : 0u;
                }
            }
        }
        __syncthreads();

        // ---- body: Genz recursion over shifts x lattice slices ----
        const int units = (s_hi - s_lo) * slices;
        if (!sm.bad && q > 0) {
            for (int un = warp; un < units; un += n_warps) {
                const int s = s_lo + un / slices, h = un % slices;
                const int64_t k0 = (Pd.N * h) / slices, k1 = (Pd.N * (h + 1)) / slices;
                double an = 0.0, ad = 0.0;
                if constexpr (MODE == kModeFast) {
                    if (c == q)  // classic term (or a group of one): no capture in the loop
                        genz_points_fast<DMAX, P, false>(sm, q, c, s, max_S, k0, k1, an, ad);
                    else
                        genz_points_fast<DMAX, P, true>(sm, q, c, s, max_S, k0, k1, an, ad);
                }
                else if constexpr (MODE == kModeSafe)
                    genz_points_safe<DMAX, P>(sm, q, c, s, k0, k1, an, ad);
                else
                    genz_points_fp64<DMAX>(sm, Pd, q, c, s, k0, k1, an, ad);
                an = warp_sum(an);
                ad = warp_sum(ad);
                if (lane == 0) {
                    sm.part_num[un] = an;
                    sm.part_den[un] = ad;
                }
            }
        }
        __syncthreads();

        // ---- epilogue: per-shift means ----
        for (int s = s_lo + threadIdx.x; s < s_hi; s += blockDim.x) {
            const int un0 = (s - s_lo) * slices;
            double vn, vd;
            if (sm.bad) {
                vn = vd = __longlong_as_double(0x7ff8000000000000LL);
            } else if (q == 0) {
                vn = sm.e0;
                vd = 1.0;
            } else {
                double sn = 0.0, sd = 0.0;
                for (int h = 0; h < slices; ++h) {
                    sn += sm.part_num[un0 + h];
                    sd += sm.part_den[un0 + h];
                }
                vn = sn / (double)Pd.N;
                vd = sd / (double)Pd.N;
                if constexpr (MIXED) {
                    vn *= sm.e0;
                    vd *= sm.e0;
                }
                if (c == 0) vd = 1.0;  // no conditioning set: the term is the joint CDF itself
                if constexpr (MIXED) {
                    // the fast form is exact to 2^-22 only for means >= 2^-40
                    if (MODE == kModeFast && !(vn >= 0x1p-40 && vd >= 0x1p-40 && isfinite(vn) && isfinite(vd)))
                        sm.flag = 1;
                }
            }
            Pd.num[term * S + s] = vn;
            Pd.den[term * S + s] = vd;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sm.bad) {
                ProbResult* R = Pd.res ? Pd.res : &results[item.x];
                atomicMin((unsigned long long*)&R->bad_site, (unsigned long long)term);
                R->status = (sm.bad == 1) ? VECCHIA_ERR_NOT_PD : VECCHIA_ERR_ARG;
            } else if (MODE == kModeFast && sm.flag && fallback_items) {
                const int pos = atomicAdd(fallback_count, 1);
                if (pos < src.fb_cap) fallback_items[pos] = item;  // the callers size it for every item
            }
        }
        __syncthreads();
    }
}

// ------------------------------- log-sum ------------------------------------
// Two passes with a fixed reduction order, so results are bit-identical run to
// run and alone vs in a batch:
//   partial: CTA (slice, problem) takes sites slice*32 .. +31, forms each
//     term T_i = log mean_s num - log mean_s den (Sec. 3.1: every term on the
//     log scale) and the delta-method pieces num_is/numbar_i - den_is/denbar_i,
//     and writes their slice sums;
//   final: one warp per problem adds the slices in order and forms
//     log P = sum_i T_i and SE = sqrt(sum_s l_s^2 / (S (S-1))).

// One warp a slice: the per-site work (two FP64 logarithms and the S
// delta-method quotients) is FP64-bound on GB300, so a 2,500-site problem is
// spread over 79 SMs rather than 10.
constexpr int kSliceSites = kLogsumSlice;

__device__ __forceinline__ double warp_sum_xor(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kSliceSites) logsum_partial_kernel(
    const ProbDev* __restrict__ probs, double* const* __restrict__ terms, double* __restrict__ scratch,
    const int64_t* __restrict__ scratch_off) {
    __shared__ double red[kMaxS + 1][kSliceSites / 32];
    const int pi = blockIdx.y, slice = blockIdx.x;
    const ProbDev& Pd = probs[pi];
    const int64_t D = Pd.n_terms;
    const int S = Pd.S;
    if ((int64_t)slice * kSliceSites >= D) return;  // CTA-uniform
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)slice * kSliceSites + tid;
    const bool valid = i < D;
    double T = 0.0, a = 1.0, b = 1.0;
    if (valid) {
        double sn = 0.0, sd = 0.0;
        for (int s = 0; s < S; ++s) {
            sn += Pd.num[i * S + s];
            sd += Pd.den[i * S + s];
        }
        a = sn / (double)S;
        b = sd / (double)S;
        T = log(a) - log(b);
        if (terms && terms[pi]) terms[pi][i] = T;
    }
    double v = warp_sum_xor(T);
    if (lane == 0) red[0][warp] = v;
    for (int s = 0; s < S; ++s) {  // quotients, not products by reciprocals: equal shifts give exactly 0
        const double c = valid ? Pd.num[i * S + s] / a - Pd.den[i * S + s] / b : 0.0;
        v = warp_sum_xor(c);
        if (lane == 0) red[1 + s][warp] = v;
    }
    __syncthreads();
    double* out = scratch + scratch_off[pi] + (int64_t)slice * (S + 1);
    for (int c = tid; c <= S; c += blockDim.x) {
        double acc = 0.0;
        for (int w = 0; w < kSliceSites / 32; ++w) acc += red[c][w];
        out[c] = acc;
    }
}

__global__ void __launch_bounds__(32) logsum_final_kernel(const ProbDev* __restrict__ probs,
                                                          ProbResult* __restrict__ results,
                                                          const double* __restrict__ scratch,
                                                          const int64_t* __restrict__ scratch_off) {
    const int pi = blockIdx.x, lane = threadIdx.x;
    const ProbDev& Pd = probs[pi];
    const int64_t D = Pd.n_terms;
    const int S = Pd.S;
    if (D <= 0 || S < 2) return;
    const int slices = (int)((D + kSliceSites - 1) / kSliceSites);
    const double* part = scratch + scratch_off[pi];
    double col[3] = {0.0, 0.0, 0.0};  // columns lane, lane + 32, lane + 64 (S + 1 <= 65)
    for (int k = 0; k < 3; ++k) {
        const int c = lane + 32 * k;
        if (c <= S)
            for (int sl = 0; sl < slices; ++sl) col[k] += part[(int64_t)sl * (S + 1) + c];
    }
    double log_p = __shfl_sync(0xffffffffu, col[0], 0);
    double ss = 0.0;
    for (int c = 1; c <= S; ++c) {
        const double l = __shfl_sync(0xffffffffu, col[c >> 5], c & 31);
        ss += l * l;
    }
    if (lane == 0) {
        ProbResult& R = Pd.res ? *Pd.res : results[pi];
        R.log_p = log_p;
        R.std_err = sqrt(ss / ((double)S * (double)(S - 1)));
        if (R.status == VECCHIA_OK && !(isfinite(log_p) && isfinite(R.std_err)))
            R.status = VECCHIA_ERR_NONFINITE;
    }
}

__global__ void init_results_kernel(ProbResult* r, int n, int* fallback_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        r[i].log_p = 0.0;
        r[i].std_err = 0.0;
        r[i].bad_site = LLONG_MAX;
        r[i].status = VECCHIA_OK;
        r[i].pad = 0;
    }
    if (i == 0 && fallback_count) *fallback_count = 0;
}

// ------------------------------- shifts -------------------------------------

__global__ void shifts_kernel(const uint64_t* __restrict__ seeds, const int32_t* __restrict__ Ss,
                              const int64_t* __restrict__ off, int n_probs, int dim,
                              double* __restrict__ delta, uint32_t* __restrict__ dfix) {
    const int pi = blockIdx.y;
    if (pi >= n_probs) return;
    const int S = Ss[pi];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= S * dim) return;
    const int s = x / dim, j = x % dim;
    uint32_t c[4] = {(uint32_t)s, (uint32_t)j, 0x51A7u, 0u};
    const uint64_t seed = seeds[pi];
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const uint64_t M = ((uint64_t)(c[0] >> 5) << 26) | (uint64_t)(c[1] >> 6);  // 53-bit integer
    delta[off[pi] + x] = (double)M * 0x1p-53;
    dfix[off[pi] + x] = (uint32_t)(M >> 21);
}

__global__ void eval_special_kernel(int which, const float* __restrict__ x, int64_t n,
                                    float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = x[i];
    float e, ec, le2 = 0.0f, r = 0.0f;
    bool tiny;
    switch (which) {
        case 0: special::phi_pair(v, e, ec, tiny, le2); r = e; break;
        case 1: special::phi_pair(v, e, ec, tiny, le2); r = ec; break;
        case 2: special::phi_pair(v, e, ec, tiny, le2); r = tiny ? le2 : NAN; break;
        case 3: r = special::phiinv_pq(v, 1.0f - v); break;
        case 4: r = special::phiinv_log2(v); break;
        case 5: special::phi_pair_fast_s(v, e, ec); r = e; break;
        case 6: special::phi_pair_fast_s(v, e, ec); r = ec; break;
        case 7: r = special::phiinv16_pq(__fmul_rn(16.0f, v), __fmul_rn(16.0f, __fsub_rn(1.0f, v))); break;
        default: r = NAN;
    }
    out[i] = r;
}

// FP64 forms of the FP64 path: which = 0: Phi(x); 1: 1 - Phi(x); 2: Phi^{-1}(x)
// given p = x and q = 1 - x; 3: Phi^{-1}(1 - x) given q = x and p = 1 - x, i.e.
// -Phi^{-1}(x) taken from the upper argument.
__global__ void eval_special64_kernel(int which, const double* __restrict__ x, int64_t n,
                                      double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char tb_smem[];
    special64::Tables64& tb = *reinterpret_cast<special64::Tables64*>(tb_smem);
    special64::load_tables(tb);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    double e, ec, r;
    switch (which) {
        case 0: special64::phi_pair(tb, v, e, ec); r = e; break;
        case 1: special64::phi_pair(tb, v, e, ec); r = ec; break;
        case 2: r = special64::phiinv_pq(tb, v, 1.0 - v); break;
        case 3: r = special64::phiinv_pq(tb, 1.0 - v, v); break;
        default: r = NAN;
    }
    out[i] = r;
}

}  // namespace

cudaError_t launch_eval_special64(int which, const double* x, int64_t n, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    eval_special64_kernel<<<(int)((n + 255) / 256), 256, sizeof(special64::Tables64), st>>>(which, x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_eval_special(int which, const float* x, int64_t n, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    eval_special_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(which, x, n, out);
    return cudaGetLastError();
}

// ------------------------------- launchers ----------------------------------

namespace {

template <int DMAX, int P, int MODE>
cudaError_t launch_one(const GenzTile& tile, const ProbDev* probs, const ItemSrc& src, int max_S,
                       ProbResult* results, int* fb_count, int2* fb_items, cudaStream_t st) {
    auto kern = genz_kernel<DMAX, P, MODE>;
    constexpr bool MIXED = MODE != kModeFP64;
    constexpr int kWarpCap = max_threads(DMAX, P, MODE) / 32;
    const int warps = tile.warps < 1 ? 1 : (tile.warps > kWarpCap ? kWarpCap : tile.warps);
    const size_t smem = smem_bytes<DMAX, MIXED>(max_S < 1 ? 1 : max_S, warps);
    int dev = 0;
    cudaGetDevice(&dev);
    // occupancy per (device, warps, shared bytes); the attribute once per device
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t>, int> per_sm;
    static std::map<int, size_t> attr_set;
    int blocks_per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto& a = attr_set[dev];
        if (smem > 48 * 1024 && a < smem) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            a = smem;
        }
        auto key = std::make_tuple(dev, warps, smem);
        auto it = per_sm.find(key);
        if (it == per_sm.end()) {
            int b = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, warps * 32, smem);
            if (e != cudaSuccess) return e;
            it = per_sm.emplace(key, b > 0 ? b : 1).first;
        }
        blocks_per_sm = it->second;
    }
    const int64_t cap = (int64_t)blocks_per_sm * device_sm_count(dev);
    ItemSrc s2 = src;
    if (!src.items && src.n_items > cap) {
        // cut the sites of the last, partial round into more shift groups (as
        // long as each piece keeps a shift per warp and the pieces fit one round)
        const int g = src.groups, n_sites = src.n_items / g;
        const int whole_sites = (int)(((int64_t)(src.n_items / cap) * cap) / g);
        const int rest = n_sites - whole_sites;
        int tg = g;
        while (rest > 0 && 2 * tg * warps <= max_S && (int64_t)rest * 2 * tg <= cap) tg *= 2;
        if (tg > g) {
            s2.whole_sites = whole_sites;
            s2.tail_groups = tg;
            s2.n_items = whole_sites * g + rest * tg;
        }
    }
    const int grid = (int)((s2.n_items < cap) ? s2.n_items : cap);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, warps * 32, smem, st>>>(probs, s2, tile.slices, max_S, results, fb_count, fb_items);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_genz(int bucket, bool mixed, const GenzTile& tile, const ProbDev* probs,
                        const int* seg_prefix, const int2* seg_base, int n_segs, int n_sites,
                        ProbResult* results, int* fallback_count, int2* fallback_items, int max_S,
                        int fb_capacity, cudaStream_t st) {
    if (n_sites <= 0) return cudaSuccess;
    GenzTile t = tile;
    if (t.slices < 1) t.slices = 1;
    if (t.groups < 1) t.groups = 1;
    if (t.groups > max_S) t.groups = max_S;
    const int per_group = (max_S + t.groups - 1) / t.groups;
    while (t.slices > 1 && per_group * t.slices > kMaxUnits) --t.slices;
    ItemSrc src{nullptr, nullptr, seg_prefix, seg_base, n_segs, n_sites * t.groups, t.groups, n_sites, t.groups,
                fb_capacity};
#define VK_ARGS t, probs, src, max_S, results
#define VK_CASE(IDX, DM)                                                                         \
    case IDX:                                                                                    \
        if (!mixed) return launch_one<DM, 1, kModeFP64>(VK_ARGS, nullptr, nullptr, st);           \
        if (t.points >= 2)                                                                       \
            return launch_one<DM, 2, kModeFast>(VK_ARGS, fallback_count, fallback_items, st);    \
        return launch_one<DM, 1, kModeFast>(VK_ARGS, fallback_count, fallback_items, st);
#define VK_CASE1(IDX, DM)                                                                        \
    case IDX:                                                                                    \
        if (!mixed) return launch_one<DM, 1, kModeFP64>(VK_ARGS, nullptr, nullptr, st);           \
        return launch_one<DM, 1, kModeFast>(VK_ARGS, fallback_count, fallback_items, st);
    static_assert(kNumBuckets == 9, "bucket table");
    switch (bucket) {
        VK_CASE(0, 9)
        VK_CASE(1, 13)
        VK_CASE(2, 17)
        VK_CASE(3, 21)
        VK_CASE(4, 25)
        VK_CASE(5, 29)
        VK_CASE(6, 32)
        VK_CASE1(7, 48)
        VK_CASE1(8, 64)
        default:
            return cudaErrorInvalidValue;
    }
#undef VK_CASE
#undef VK_CASE1
#undef VK_ARGS
}

cudaError_t launch_genz_fallback(int max_bucket, const ProbDev* probs, const int* fallback_count,
                                 const int2* fallback_items, int capacity, ProbResult* results,
                                 int max_S, cudaStream_t st) {
    if (capacity <= 0) return cudaSuccess;
    GenzTile t{4, 1, 1, 1};
    ItemSrc src{fallback_items, fallback_count, nullptr, nullptr, 0, capacity, 1, 0, 1, 0};
    if (max_bucket >= 7)  // blocks of more than 32 variables in the batch
        return launch_one<64, 1, kModeSafe>(t, probs, src, max_S, results, nullptr, nullptr, st);
    return launch_one<32, 1, kModeSafe>(t, probs, src, max_S, results, nullptr, nullptr, st);
}

cudaError_t launch_logsum(const ProbDev* probs, int n_probs, int max_slices, ProbResult* results,
                          double* const* terms, double* scratch, const int64_t* scratch_off,
                          cudaStream_t st) {
    if (n_probs <= 0 || max_slices <= 0) return cudaSuccess;
    logsum_partial_kernel<<<dim3(max_slices, n_probs), kSliceSites, 0, st>>>(probs, terms, scratch,
                                                                          scratch_off);
    logsum_final_kernel<<<n_probs, 32, 0, st>>>(probs, results, scratch, scratch_off);
    return cudaGetLastError();
}

cudaError_t launch_shifts(const uint64_t* seeds, const int32_t* S, const int64_t* out_off,
                          int n_probs, int dim, double* delta, uint32_t* dfix, cudaStream_t st) {
    if (n_probs <= 0 || dim <= 0) return cudaSuccess;
    const int per = kMaxS * dim;
    dim3 grid((per + 127) / 128, n_probs);
    shifts_kernel<<<grid, 128, 0, st>>>(seeds, S, out_off, n_probs, dim, delta, dfix);
    return cudaGetLastError();
}

cudaError_t launch_init_results(ProbResult* results, int n, int* fallback_count, cudaStream_t st) {
    const int nn = n > 1 ? n : 1;
    init_results_kernel<<<(nn + 255) / 256, 256, 0, st>>>(results, n, fallback_count);
    return cudaGetLastError();
}

}  // namespace vk
