// full_tc.cu -- the mixed-precision full D-dimensional Genz estimate (Sec. 2.2,
// Sec. 3: the m = D - 1 limit of Eq. vecchia-cdf) with the history
// contraction on the tensor cores: tcgen05.mma with TF32 operands staged in
// shared memory and FP32 accumulators in tensor memory.
//
// For a CTA tile of 224 lattice points (row blocks of M = 128: all 128 rows of
// the first, 96 of the second) and a panel of 64 variables v0 .. v0+63, the
// panel's conditional means need
//     acc[p][j] = sum_{t < v0} y_t[p] Ls[v0 + j][t],
// a dense (points x t) by (t x variables) product over the stored y history.
// Each FP32 operand x is split as x = hi + lo, hi = x rounded to TF32 (11
// significant bits, to nearest) and lo = the remainder rounded likewise, and
// the product is taken as hi.hi + hi.lo + lo.hi: the dropped lo.lo term and the
// rounding of lo are each below 2^-22 of |x y|, near FP32's own rounding.
//
// Roles (256 threads: seven point warps and one copy/MMA warp, so that two
// CTAs per SM leave four warps and 128 registers a thread on each SMSP):
//   warp 7 lane 0 streams history chunks (16 variables x 224 points, hi and lo,
//     28 KB) and the matching blocks of L (64 x 16, hi and lo, 8 KB each)
//     through a two-stage shared-memory ring with cp.async.bulk and issues the
//     MMAs.  Panels go in pairs (b, b + 1): one pass over the history chunks
//     below panel b feeds both panels' accumulators (24 MMAs a chunk), so the
//     history is read once per pair; the four chunks of panel b's own y then
//     complete panel b + 1.  A chunk is loaded only after the point threads
//     have written it;
//   warps 0..6, one thread per point, run each panel's variables in order from
//     the accumulator: the in-panel terms (FP32 fma, right-looking), Phi, the
//     running product in FP64, Phi^{-1} of the lattice-weighted probability;
//     y goes to the history (hi, lo) in the MMA operand layout.
// The two accumulators of a pair fill the CTA's 256 tensor-memory columns; the
// next pair's MMAs start once panel b + 1's accumulator has been read out, so
// they run while panel b + 1's variables are processed.  Every wait is bounded
// by the global timer; on expiry the kernel records a timeout, waits (bounded)
// for its copies and MMAs in flight, frees its tensor memory and returns.  The
// limit of the point warps' waits and of the copy lane's idle time can be set
// shorter (for tests); the drain waits keep the full 2 s, so whatever was
// issued completes before the tensor memory is freed.  For the timeout test,
// the copy lane can be told to issue nothing: then the first accumulator wait
// of the point warps runs out with no copy and no MMA in flight.
//
// Operand layout (no swizzle, K-major): 8-row x 16-byte core matrices; within
// a block, element (r, k) of a 16-wide chunk sits at byte
//     (r / 8) * 512 + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4,
// so the descriptor's K-direction core-matrix stride is 128 B and its
// row-group stride 512 B.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "special_f32.h"
#include "vk_internal.h"

namespace vk {
namespace {

constexpr int kTcPoints = 224;                  // lattice points per CTA (rows 0..223 of 256)
constexpr int kTcHalf = 128;                    // MMA M
constexpr int kTcB = 64;                        // panel width = MMA N
constexpr int kTcKC = 16;                       // history chunk (variables)
constexpr int kTcStages = 2;
constexpr int kTcThreads = kTcPoints + 32;      // point warps + the copy/MMA warp
constexpr uint32_t kChunkA = 2 * kTcHalf * kTcKC * 4 * 2;  // 32 KB: y hi, y lo (256 rows)
constexpr uint32_t kRowsA = kTcPoints * kTcKC * 4;          // 14 KB: the used rows of hi (or lo)
constexpr uint32_t kChunkB = kTcB * kTcKC * 4 * 2;       // 8 KB: L hi, L lo
constexpr uint32_t kStageA = 2 * kRowsA;                    // 28 KB: y hi, then y lo (224 rows each)
constexpr uint32_t kStageBytes = kStageA + 2 * kChunkB;      // + the L blocks of a pair's two panels
constexpr uint32_t kLpBytes = kTcB * kTcB * 4;           // the panel's own triangle
constexpr uint32_t kPanBytes = 3 * kTcB * 4;                 // the panel's us, g, Delta_s (one shift per CTA)
constexpr uint32_t kTcSmem = kTcStages * kStageBytes + kLpBytes + kPanBytes;
constexpr uint32_t kTmemCols = 2 * 2 * kTcB;             // 2 panels x 2 row blocks x 64
constexpr uint64_t kWaitNs = 2000000000ull;              // 2 s without progress

// instruction descriptor: D F32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcB >> 3) << 17) |
                            ((uint32_t)(kTcHalf >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking test of the phase of the given parity (for a thread that polls
// several barriers in turn).
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns = kWaitNs) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try(b, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// shared-memory matrix descriptor: no swizzle, K stride 128 B, row-group stride 512 B
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
           ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// OR of a predicate over the 224 point threads (named barrier 1)
__device__ __forceinline__ bool points_any(bool q) {
    uint32_t r;
    asm volatile("{\n .reg .pred q, r;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred r, 1, 224, q;\n selp.u32 %0, 1, 0, r;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)q)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ void points_sync() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

// x rounded to the nearest TF32 value (ties away from zero): add half a unit of
// the 13 dropped bits to the magnitude and clear them.
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

struct TcArgs {
    int D, Dp, nP, nC;          // variables, padded to 64, panels, chunks of 16
    int64_t N;
    int S, tps;                 // tiles per shift (224 points)
    int dim;                    // row stride of dfix
    const uint32_t* gfix;       // round(g 2^32 / N)
    const uint32_t* dfix;       // S x dim shift tables (top 32 bits)
    const float* us;            // u_v / L_vv, padded with 0
    const float* Lb;            // blocked L/diag, hi and lo, [nP][nC] blocks of 8 KB
    const float* LpT;           // [nP][64][64]: LpT[j][j'] = Ls[v0 + j'][v0 + j], j < j'
    float* Y;                   // history, [tiles][nC] chunks of 32 KB
    double* part;               // per shift, per tile: sums over points 0..127 and 128..223
    int* timeout;               // set on an expired wait
    uint64_t wait_ns;           // limit of the point warps' waits and of the copy lane's idle time
    int withhold;               // testing: the copy lane issues no copy and no MMA
};

// Tables of the scaled factor for the tensor-core path: the blocked hi/lo
// operand Lb (rows of panel b, columns t < 64 b), the in-panel triangle LpT
// and us.  Ls = L_vt / L_vv in FP64, rounded to FP32 (as the FP32 path).
__global__ void tc_tables_kernel(const double* __restrict__ A, const double* __restrict__ u, int D, int Dp, int nC,
                                 float* __restrict__ Lb, float* __restrict__ LpT, float* __restrict__ us) {
    const int v = blockIdx.y, b = v / kTcB, r = v % kTcB, v0 = b * kTcB;
    const double rd = (v < D) ? 1.0 / A[(int64_t)v * D + v] : 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < v; t += gridDim.x * blockDim.x) {
        const float x = (v < D) ? (float)(A[(int64_t)v * D + t] * rd) : 0.0f;
        if (t < v0) {
            const int c = t / kTcKC, kk = t % kTcKC;
            const int64_t off = ((int64_t)b * nC + c) * (kChunkB / 4) + (r / 8) * 128 + (kk / 4) * 32 + (r % 8) * 4 +
                                (kk % 4);
            const float hi = tf32_round(x);
            Lb[off] = hi;
            Lb[off + kChunkB / 8] = tf32_round(x - hi);
        } else {
            LpT[(int64_t)b * kTcB * kTcB + (t - v0) * kTcB + r] = x;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) us[v] = (v < D) ? (float)(u[v] * rd) : 0.0f;
}

// One variable of one point: e = Phi(z) and, if wanted, y = Phi^{-1}(w e) at
// the lattice coordinate X = k g_v + Delta_v (32-bit fixed point).  Kept out
// of line so that the panel loop around it unrolls with its accumulators in
// registers.
__device__ __noinline__ float2 tc_phi_y(float z, uint32_t X, bool want_y) {
    float e, ec;
    special::phi_pair_fast(z, e, ec);
    float y = 0.0f;
    if (want_y) {
        const uint32_t V = ((int32_t)X < 0) ? 0u - X : X;  // tent: w = |int32(X)| 2^-31
        const float w = __fmul_rn(__uint2float_rn(V), 0x1p-31f);
        const float am = __fmul_rn(__uint2float_rn(0x80000000u - V), 0x1p-31f);  // |2x - 1|
        y = special::phiinv_pq(__fmul_rn(w, e), fmaf(w, ec, am));
    }
    return make_float2(e, y);
}

// Jobs (history chunks) of pair q = panels 2q and 2q + 1 of nP.
__device__ __forceinline__ int pair_jobs(int q, int nP) {
    const int b = 2 * q;
    return 4 * b + (b + 1 < nP ? 4 : 0);
}
// Move a (pair, job) cursor past finished pairs.
__device__ __forceinline__ void skip_empty_pairs(int& q, int& c, int nQ, int nP) {
    while (q < nQ && c >= pair_jobs(q, nP)) {
        c = 0;
        ++q;
    }
}

// The state one point thread carries through a panel.
struct PanelState {
    float* z;         // [64] conditional sums of the panel's variables (registers)
    float yh[4], yl[4];
    double f;         // running product
    int nb, v0;
    uint32_t k;       // lattice point index
    float* Yp;        // this point's slot in the history layout
    const float* Lp;  // the panel's triangle, LpT[j][j'] (shared memory)
    const float* us;  // the panel's u_v / L_vv (shared memory)
    const uint32_t* gd;  // the panel's lattice g (64 entries), then the CTA's shift (64)
};

// Variable J of the panel: e and y, the in-panel terms of the later variables
// (right-looking), y (hi, lo) to the history every four variables.
template <int J>
__device__ __forceinline__ void panel_step(const TcArgs& a, PanelState& ps) {
    if (J >= ps.nb) return;
    const int v = ps.v0 + J;
    const bool want_y = v < a.D - 1;
    const uint32_t X = ps.k * ps.gd[J] + ps.gd[kTcB + J];
    const float2 ey = tc_phi_y(__fsub_rn(ps.us[J], ps.z[J]), X, want_y);
    ps.f *= (double)ey.x;
    const float y = ey.y, hi = tf32_round(y);
    ps.yh[J % 4] = hi;
    ps.yl[J % 4] = tf32_round(__fsub_rn(y, hi));
    const float* row = ps.Lp + J * kTcB;
#pragma unroll
    for (int jp = J + 1; jp < kTcB; ++jp) ps.z[jp] = fmaf(row[jp], y, ps.z[jp]);
    if (J % 4 == 3) {
        float* dst = ps.Yp + (int64_t)(v / kTcKC) * (kChunkA / 4) + ((J % kTcKC) / 4) * 32;
        *(float4*)dst = make_float4(ps.yh[0], ps.yh[1], ps.yh[2], ps.yh[3]);
        *(float4*)(dst + kChunkA / 8) = make_float4(ps.yl[0], ps.yl[1], ps.yl[2], ps.yl[3]);
    }
}
template <int... J>
__device__ __forceinline__ void panel_steps(const TcArgs& a, PanelState& ps, std::integer_sequence<int, J...>) {
    (panel_step<J>(a, ps), ...);
}

__global__ void __launch_bounds__(kTcThreads, 2) full_genz_tc_kernel(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar_full[kTcStages], bar_empty[kTcStages], bar_acc[2], bar_ydone, bar_tfree;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ double red[kTcPoints / 32];
    float* sLp = (float*)(tc_smem + kTcStages * kStageBytes);
    float* sUs = sLp + kTcB * kTcB;               // [64] us of the panel
    uint32_t* sGD = (uint32_t*)(sUs + kTcB);      // [64] g, [64] Delta of this CTA's shift
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x, s = tile / a.tps, tile_in_shift = tile % a.tps;
    float* Yt = a.Y + (int64_t)tile * a.nC * (kChunkA / 4);

    if (warp == 7) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            mbar_init(&bar_full[i], 1);
            mbar_init(&bar_empty[i], 1);
        }
        mbar_init(&bar_acc[0], 1);
        mbar_init(&bar_acc[1], 1);
        mbar_init(&bar_ydone, kTcPoints);
        mbar_init(&bar_tfree, kTcPoints);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int nP = a.nP;

    if (warp == 7) {
        if (lane == 0) {
            // ---- copies and MMAs, pair by pair: pair q = panels b = 2q and b + 1 ----
            // job c of a pair is history chunk c: chunks c < 4b feed both panels
            // (shared), chunks 4b .. 4b+3 (panel b's y) only panel b + 1 (own)
            const int nQ = (nP + 1) / 2;
            int total = 0;
            for (int q = 0; q < nQ; ++q) total += pair_jobs(q, nP);
            int il = 0, lq = 0, lc = 0;  // next load: pair, job
            int im = 0, mq = 0, mc = 0;  // next MMA
            skip_empty_pairs(lq, lc, nQ, nP);
            skip_empty_pairs(mq, mc, nQ, nP);
            int seen = 0;   // panels whose y the point threads have written
            int freed = 0;  // pairs whose accumulators the point threads have read
            bool failed = false;
            uint64_t t_idle = 0;
            int spins = 0;
            while (im < total) {
                bool progress = false;
                if (il < total && il < im + kTcStages && !a.withhold) {
                    const int b = 2 * lq, c = lc;
                    const bool shared = c < 4 * b, has2 = b + 1 < nP;
                    bool gate = true;
                    if (seen <= c / 4) {  // chunk c holds panel c / 4's y
                        if (mbar_test(&bar_ydone, (uint32_t)(seen & 1))) ++seen;
                        gate = seen > c / 4;
                    }
                    const int st = il % kTcStages;
                    const uint32_t par = (uint32_t)(((il / kTcStages) & 1) ^ 1);
                    if (gate && mbar_test(&bar_empty[st], par)) {
                        unsigned char* sA = tc_smem + st * kStageBytes;
                        const float* ysrc = Yt + (int64_t)c * (kChunkA / 4);
                        const uint32_t nl = (shared && has2) ? 2u : 1u;
                        mbar_expect_tx(&bar_full[st], kStageA + nl * kChunkB);
                        bulk_g2s(sA, ysrc, kRowsA, &bar_full[st]);
                        bulk_g2s(sA + kRowsA, ysrc + kChunkA / 8, kRowsA, &bar_full[st]);
                        if (shared)
                            bulk_g2s(sA + kStageA, a.Lb + ((int64_t)b * a.nC + c) * (kChunkB / 4), kChunkB,
                                     &bar_full[st]);
                        if (has2)
                            bulk_g2s(sA + kStageA + kChunkB, a.Lb + ((int64_t)(b + 1) * a.nC + c) * (kChunkB / 4),
                                     kChunkB, &bar_full[st]);
                        ++il;
                        ++lc;
                        skip_empty_pairs(lq, lc, nQ, nP);
                        progress = true;
                    }
                }
                if (im < il) {
                    const int b = 2 * mq, c = mc;
                    const bool shared = c < 4 * b, has2 = b + 1 < nP;
                    bool gate = true;
                    if (mq >= 1 && freed < mq) {  // the previous pair's accumulators read out
                        if (mbar_test(&bar_tfree, (uint32_t)((mq - 1) & 1)))
                            freed = mq;
                        else
                            gate = false;
                    }
                    const int st = im % kTcStages;
                    if (gate && mbar_test(&bar_full[st], (uint32_t)((im / kTcStages) & 1))) {
                        tc_fence_after();
                        const uint32_t sA = smem_u32(tc_smem + st * kStageBytes);
                        const uint32_t sB0 = sA + kStageA, sB1 = sB0 + kChunkB;
#pragma unroll
                        for (int ks = 0; ks < kTcKC / 8; ++ks) {
                            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const uint64_t ah = sdesc(sA + h * (kChunkA / 4) + ks * 256);
                                const uint64_t al = sdesc(sA + kRowsA + h * (kChunkA / 4) + ks * 256);
                                if (shared) {
                                    const uint32_t d = tmem + (uint32_t)(h * kTcB);
                                    const uint64_t bh = sdesc(sB0 + ks * 256), bl = sdesc(sB0 + kChunkB / 2 + ks * 256);
                                    mma_tf32(d, ah, bh, acc);
                                    mma_tf32(d, ah, bl, 1u);
                                    mma_tf32(d, al, bh, 1u);
                                }
                                if (has2) {
                                    const uint32_t d = tmem + (uint32_t)(2 * kTcB + h * kTcB);
                                    const uint64_t bh = sdesc(sB1 + ks * 256), bl = sdesc(sB1 + kChunkB / 2 + ks * 256);
                                    mma_tf32(d, ah, bh, acc);
                                    mma_tf32(d, ah, bl, 1u);
                                    mma_tf32(d, al, bh, 1u);
                                }
                            }
                        }
                        mma_commit(&bar_empty[st]);
                        if (shared && c == 4 * b - 1) mma_commit(&bar_acc[0]);
                        if (!shared && c == 4 * b + 3) mma_commit(&bar_acc[1]);
                        ++im;
                        ++mc;
                        skip_empty_pairs(mq, mc, nQ, nP);
                        progress = true;
                    }
                }
                if (progress) {
                    spins = 0;
                    t_idle = 0;
                } else {
                    __nanosleep(32);  // leave the issue slots to the point warps
                    if (++spins == 64) {
                        spins = 0;
                        const uint64_t now = global_ns();
                        if (t_idle == 0) {
                            t_idle = now;
                        } else if (now - t_idle > a.wait_ns || *(volatile int*)&abort_flag) {
                            failed = true;
                            break;
                        }
                    }
                }
            }
            if (failed) {
                atomicExch(&abort_flag, 1);
                atomicExch(a.timeout, 1);
            }
            // copies in flight and the last MMAs, bounded
            for (int i = im; i < il; ++i) mbar_wait(&bar_full[i % kTcStages], (uint32_t)((i / kTcStages) & 1));
            if (im > 0) mbar_wait(&bar_empty[(im - 1) % kTcStages], (uint32_t)(((im - 1) / kTcStages) & 1));
        }
    } else {
        // ---- one thread per lattice point ----
        const int p = tid, h = warp >> 2, q = warp & 3;
        const int64_t k64 = (int64_t)tile_in_shift * kTcPoints + p;
        const bool valid = k64 < a.N;
        const uint32_t k = (uint32_t)(valid ? k64 : a.N - 1);
        const int r = p % kTcHalf;
        float* Yp = Yt + h * (kChunkA / 16) + (r / 8) * 128 + (r % 8) * 4;  // + chunk, + hi/lo, + k-group
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * kTcB);
        double f = 1.0;
        for (int b = 0; b < nP; ++b) {
            const int v0 = b * kTcB, nb = min(kTcB, a.D - v0);
            bool ok = true;
            // panel 2q: the shared chunks of pair q (q >= 1); panel 2q + 1: its own chunks too
            if (b > 0)
                ok = (b & 1) ? mbar_wait(&bar_acc[1], (uint32_t)((b >> 1) & 1), a.wait_ns)
                             : mbar_wait(&bar_acc[0], (uint32_t)(((b >> 1) - 1) & 1), a.wait_ns);
            if (points_any(!ok || *(volatile int*)&abort_flag)) {
                if (p == 0) {
                    atomicExch(&abort_flag, 1);
                    atomicExch(a.timeout, 1);
                }
                break;
            }
            {
                const float4* src = (const float4*)(a.LpT + (int64_t)b * kTcB * kTcB);
                for (int i = p; i < kTcB * kTcB / 4; i += kTcPoints) ((float4*)sLp)[i] = __ldg(src + i);
                if (p < kTcB) {
                    sUs[p] = __ldg(a.us + v0 + p);  // padded to a multiple of 64
                } else if (p < 3 * kTcB) {
                    const int j = (p - kTcB) % kTcB, v = v0 + j;  // g and Delta exist for v < D - 1
                    sGD[p - kTcB] = (v < a.dim) ? (p < 2 * kTcB ? __ldg(a.gfix + v) : __ldg(a.dfix + (int64_t)s * a.dim + v))
                                                : 0u;
                }
            }
            float z[kTcB];
            if (b > 0) {
                tc_fence_after();
                const uint32_t tb = tl + (uint32_t)((b & 1) * 2 * kTcB);
#pragma unroll
                for (int i = 0; i < kTcB / 16; ++i) tmem_ld16(tb + i * 16, z + 16 * i);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                tc_fence_before();
                if (b & 1) mbar_arrive(&bar_tfree);  // the pair's accumulators may be reused
            } else {
#pragma unroll
                for (int i = 0; i < kTcB; ++i) z[i] = 0.0f;
            }
            points_sync();
            PanelState ps{z, {}, {}, f, nb, v0, k, Yp, sLp, sUs, sGD};
            panel_steps(a, ps, std::make_integer_sequence<int, kTcB>{});
            f = ps.f;
            asm volatile("fence.proxy.async.global;" ::: "memory");
            mbar_arrive(&bar_ydone);
        }
        // per-128-point block sums of the point products, fixed order
        double v = valid ? f : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp] = v;
        points_sync();
        if (p == 0 || p == kTcHalf) {  // blocks of 128 and 96 points
            double t = 0.0;
            for (int w = h * 4; w < min(h * 4 + 4, kTcPoints / 32); ++w) t += red[w];
            a.part[(int64_t)s * 2 * a.tps + 2 * tile_in_shift + h] = t;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 7)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

int64_t full_tc_blocks_per_shift(int64_t N) { return 2 * ((N + kTcPoints - 1) / kTcPoints); }

size_t full_tc_scratch_bytes(int64_t D, int64_t N, int S) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int64_t Dp = (D + kTcB - 1) / kTcB * kTcB, nP = Dp / kTcB, nC = Dp / kTcKC;
    const int64_t tiles = (int64_t)S * ((N + kTcPoints - 1) / kTcPoints);
    return al((size_t)nP * nC * kChunkB) + al((size_t)nP * kLpBytes) + al(sizeof(float) * Dp) +
           al((size_t)tiles * nC * kChunkA);
}

cudaError_t launch_full_genz_tc(const double* A, const double* u, int64_t D, int64_t N, int S, const uint32_t* gfix,
                                const uint32_t* dfix, int dim, void* scratch, double* part, int* timeout,
                                uint64_t wait_ns, int withhold, cudaEvent_t ev_begin, cudaEvent_t ev_end,
                                cudaStream_t st) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int64_t Dp = (D + kTcB - 1) / kTcB * kTcB, nP = Dp / kTcB, nC = Dp / kTcKC;
    const int64_t tps = (N + kTcPoints - 1) / kTcPoints;
    char* p = (char*)scratch;
    float* Lb = (float*)p;
    p += al((size_t)nP * nC * kChunkB);
    float* LpT = (float*)p;
    p += al((size_t)nP * kLpBytes);
    float* us = (float*)p;
    p += al(sizeof(float) * Dp);
    float* Y = (float*)p;
    cudaError_t e = cudaMemsetAsync(LpT, 0, (size_t)nP * kLpBytes, st);
    if (e != cudaSuccess) return e;
    tc_tables_kernel<<<dim3((unsigned)std::min<int64_t>((Dp + 255) / 256, 8), (unsigned)Dp), 256, 0, st>>>(
        A, u, (int)D, (int)Dp, (int)nC, Lb, LpT, us);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::map<int, bool> attr;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr[dev]) {
            e = cudaFuncSetAttribute(full_genz_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
    }
    TcArgs a;
    a.D = (int)D;
    a.Dp = (int)Dp;
    a.nP = (int)nP;
    a.nC = (int)nC;
    a.N = N;
    a.S = S;
    a.tps = (int)tps;
    a.dim = dim;
    a.gfix = gfix;
    a.dfix = dfix;
    a.us = us;
    a.Lb = Lb;
    a.LpT = LpT;
    a.Y = Y;
    a.part = part;
    a.timeout = timeout;
    a.wait_ns = (wait_ns > 0 && wait_ns < kWaitNs) ? wait_ns : kWaitNs;
    a.withhold = withhold ? 1 : 0;
    if (ev_begin && (e = cudaEventRecord(ev_begin, st)) != cudaSuccess) return e;
    full_genz_tc_kernel<<<(unsigned)(S * tps), kTcThreads, kTcSmem, st>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev_end) e = cudaEventRecord(ev_end, st);
    return e;
}

}  // namespace vk
