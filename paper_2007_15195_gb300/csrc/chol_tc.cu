// chol_tc.cu -- the trailing update of the blocked Cholesky factor behind the
// mixed-precision full D-dimensional estimate (Sec. 2.2, Sec. 3: the factor
// of the whole covariance that Genz's recursion runs on), on the tensor cores
// at FP64 accuracy.
//
// Block column k (32 columns) of the factor updates the trailing matrix:
//     A_rc -= sum_{t < 32} L_rt L_ct,   r >= c >= base = 32 (k + 1).
// GB300 runs FP64 at 2 lanes per SM per clock, so this update, D^3/6 FMAs in
// all, bounds an FP64 factor.  Here each row r of the panel is written as
//     L_rt = 2^e_r x_rt,  x_rt = sum_{i < 7} s_i,rt 2^(-8 (i + 1)),
// e_r the exponent of the row's largest entry (|x| < 1) and s_i small
// integers (|s_0| <= 256, |s_i| <= 128: balanced base-256 digits of
// round(x 2^56)), each exact in bf16.  A product of two digit matrices over
// the 32 columns has integer entries below 2^21, and the products of one
// significance g = i + j (at most 7 of them) sum below 2^24: the tensor core's
// FP32 accumulation of
//     G_g = sum_{i + j = g} s_i s_j^T,   g = 0 .. 6,
// is exact.  The 28 products (two K = 16 steps each) go into seven
// accumulators in tensor memory; per entry
//     V = G_0 2^40 + G_1 2^32 + ... + G_5 + floor(G_6 / 2^8)
// is formed exactly in 64-bit integers, and
//     A_rc = fma(-(double) V, 2^(e_r + e_c - 56), A_rc),
// one rounding of V to 53 bits and one of the update: the dropped digit
// products (i + j >= 7) and digits beyond the seventh are below 2^-53 of
// sum_t |L_rt L_ct|, against 32 roundings of the FP64 fma chain.  It differs
// from the row-by-row definition in the last bits of the factor, which the
// mixed path rounds to TF32 pairs anyway; the FP64 path keeps the FP64 update.
//
// Operand layout (no swizzle, K-major): 8-row x 16-byte core matrices; the
// slice buffer of a panel holds, per group of 8 rows, the 7 digit matrices of
// those rows (512 B each: byte (k / 8) 128 + (r % 8) 16 + (k % 8) 2), so a
// tile of 128 (or 32) consecutive rows is one contiguous block: the
// descriptor's K-direction core-matrix stride is 128 B and its row-group
// stride 3,584 B.  One CTA per output tile of 128 rows x 32 columns: thread 0
// copies both operands with cp.async.bulk and issues the MMAs, the four warps
// read their 32 rows of the accumulators back.  Waits are bounded by the
// global timer; on expiry the kernel records a timeout, waits (bounded) for
// what it issued, frees its tensor memory and returns.
#include <algorithm>
#include <map>
#include <mutex>

#include "vk_internal.h"

namespace vk {
namespace {

constexpr int kTM = 128, kTN = 32;                                  // output tile
constexpr uint32_t kABytes = (kTM / 8) * kCholSliceGroupBytes;      // 57,344
constexpr uint32_t kBBytes = (kTN / 8) * kCholSliceGroupBytes;      // 14,336
constexpr uint32_t kTmemCols = 256;                                 // 7 x 32 used
// dynamic shared memory a CTA asks for: the operands, rounded up so that no
// more than two CTAs (2 x 256 tensor-memory columns) share an SM
constexpr uint32_t kSmemBytes = 80 * 1024;
static_assert(kABytes + kBBytes <= kSmemBytes, "operands fit");
constexpr uint64_t kDrainNs = 2000000000ull;

// instruction descriptor: D F32, A and B BF16, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try(b, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
// shared-memory matrix descriptor: no swizzle, K stride 128 B, row-group stride 3,584 B
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)(kCholSliceGroupBytes >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Tile (R, Cb) of the trailing matrix (rows base + 128 R .., columns
// base + 32 Cb ..): part 0 the first column block (R = blockIdx.x) below its
// diagonal block (which the factor of that block updates itself), part 1 the
// lower tiles with Cb >= 1 in row-major order (Cb <= 4 R + 3).
__device__ __forceinline__ void tile_of(int part, int nCb, int& R, int& Cb) {
    int idx = blockIdx.x;
    if (part == 0) {
        R = idx;
        Cb = 0;
        return;
    }
    for (R = 0;; ++R) {
        const int cnt = min(4 * R + 3, nCb - 1);
        if (idx < cnt) {
            Cb = 1 + idx;
            return;
        }
        idx -= cnt;
    }
}

__global__ void __launch_bounds__(128, 1) chol_update_tc_kernel(const unsigned char* __restrict__ sl,
                                                             const int* __restrict__ ex, double* __restrict__ A,
                                                             int D, int base, int part, int* timeout,
                                                             uint64_t wait_ns) {
    extern __shared__ __align__(1024) unsigned char ct_smem[];
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = D - base, nCb = (n + kTN - 1) / kTN;
    int R, Cb;
    tile_of(part, nCb, R, Cb);
    unsigned char* sA = ct_smem;
    unsigned char* sB = ct_smem + kABytes;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_load)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)) : "memory");
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (tid == 0) {
        const unsigned char* gA = sl + (size_t)R * (kTM / 8) * kCholSliceGroupBytes;
        const unsigned char* gB = sl + (size_t)Cb * (kTN / 8) * kCholSliceGroupBytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_load)),
                     "r"(kABytes + kBBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(sA)),
            "l"(gA), "r"(kABytes), "r"(smem_u32(&bar_load))
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(sB)),
            "l"(gB), "r"(kBBytes), "r"(smem_u32(&bar_load))
            : "memory");
        if (mbar_wait(&bar_load, 0, wait_ns)) {
            tc_fence_after();
            // G_g = sum_{i + j = g} s_i s_j^T, two K = 16 steps per product
#pragma unroll
            for (int g = 0; g < kCholSlices; ++g) {
                bool first = true;
#pragma unroll
                for (int i = 0; i <= g; ++i) {
                    const int j = g - i;
#pragma unroll
                    for (int kc = 0; kc < 2; ++kc) {
                        const uint64_t a = sdesc(smem_u32(sA + i * 512 + kc * 256));
                        const uint64_t b = sdesc(smem_u32(sB + j * 512 + kc * 256));
                        mma_bf16(tmem + (uint32_t)(g * kTN), a, b, first ? 0u : 1u);
                        first = false;
                    }
                }
            }
        } else {
            atomicExch(timeout, 1);
            abort_flag = 1;
            mbar_wait(&bar_load, 0, kDrainNs);  // the copies land before the CTA's memory is released
        }
        // arrives once every MMA issued above has completed (at once if none)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_mma))
                     : "memory");
    }
    __syncwarp();
    // this thread's row of the output tile, loaded while the copies and MMAs
    // run (the epilogue would otherwise wait on L2 or HBM for each chunk)
    const int r = base + R * kTM + warp * 32 + lane;
    const int c0 = base + Cb * kTN;
    double Cv[kTN];
    if (r < D) {
        const double* row = A + (int64_t)r * D + c0;
#pragma unroll
        for (int j = 0; j < kTN; ++j) Cv[j] = (c0 + j <= r) ? row[j] : 0.0;
    }
    if (!mbar_wait(&bar_mma, 0, wait_ns)) {
        atomicExch(timeout, 1);
        abort_flag = 1;
        mbar_wait(&bar_mma, 0, kDrainNs);  // the MMAs finish before the tensor memory is freed
    }
    tc_fence_after();
    __syncthreads();
    if (!abort_flag) {  // CTA-uniform: the tensor-memory loads below are warp-collective
        const int er = (r < D) ? ex[r - base] : 0;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int ch = 0; ch < kTN / 8; ++ch) {
            uint32_t G[kCholSlices][8];
#pragma unroll
            for (int g = 0; g < kCholSlices; ++g) tmem_ld8(trow + (uint32_t)(g * kTN + ch * 8), G[g]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < D) {
                double* row = A + (int64_t)r * D;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = c0 + ch * 8 + j;
                    if (c > r || (part == 0 && r < base + kTN)) continue;  // part 0: not the diagonal block
                    // exact integers below 2^24 held as FP32
                    long long V = (long long)__float2int_rz(__uint_as_float(G[0][j]));
#pragma unroll
                    for (int g = 1; g < kCholSlices - 1; ++g)
                        V = V * 256 + (long long)__float2int_rz(__uint_as_float(G[g][j]));
                    V += (long long)__float2int_rz(__uint_as_float(G[kCholSlices - 1][j])) >> 8;
                    const int e2 = er + ex[c - base] - 56;
                    if (e2 < -1020) continue;  // below 2^-1000 of the entries: nothing to subtract
                    const double scale = __hiloint2double((e2 + 1023) << 20, 0);
                    row[c] = fma(-(double)V, scale, Cv[ch * 8 + j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t chol_tc_slice_bytes(int64_t D) {
    // rows of a panel's trailing part, padded to whole tiles of 128 rows
    const int64_t groups = (D + kTM - 1) / kTM * (kTM / 8) + kTM / 8;
    return (size_t)groups * kCholSliceGroupBytes;
}

cudaError_t chol_tc_prepare() {
    static std::mutex mu;
    static std::map<int, bool> attr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(chol_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    return cudaSuccess;
}

cudaError_t launch_chol_update_tc(const unsigned char* sl, const int* ex, double* A, int64_t D, int64_t base,
                                  int part, int* timeout, uint64_t wait_ns, cudaStream_t st) {
    const int64_t n = D - base;
    if (n <= 0) return cudaSuccess;
    if (wait_ns == 0 || wait_ns > kDrainNs) wait_ns = kDrainNs;
    cudaError_t e = chol_tc_prepare();
    if (e != cudaSuccess) return e;
    const int64_t nR = (n + kTM - 1) / kTM, nCb = (n + kTN - 1) / kTN;
    int64_t tiles = 0;
    if (part == 0) {
        tiles = nR;
    } else {
        for (int64_t R = 0; R < nR; ++R) tiles += std::min<int64_t>(4 * R + 3, nCb - 1);
    }
    if (tiles <= 0) return cudaSuccess;
    chol_update_tc_kernel<<<(unsigned)tiles, 128, kSmemBytes, st>>>(sl, ex, A, (int)D, (int)base, part, timeout,
                                                                    wait_ns);
    return cudaGetLastError();
}

}  // namespace vk
