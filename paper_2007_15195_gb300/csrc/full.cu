// full.cu -- the full D-dimensional Genz estimate of P(X < u): Genz's
// separation-of-variables recursion over all D variables at the same lattice
// points and shifts as the Vecchia terms (Sec. 2.2, Sec. 3).  It is the
// m = D - 1 limit of Eq. (vecchia-cdf) (Eq. cascading-conditional-cdf
// telescopes), the estimate the Vecchia approximation is compared against.
//
//   1. covariance Sigma (FP64, lower triangle of a D x D row-major array);
//   2. Cholesky factor, blocked right-looking in FP64: a factor of each
//      32 x 32 diagonal block, a row-wise forward substitution of the rows
//      below it, and the trailing update.  Every entry receives its terms in
//      ascending k with fma and the pivot division last: the operations of
//      the row-by-row definition in its order;
//   3. the rows of L scaled by 1/L_vv (u likewise);
//   4. Genz's recursion.  FP64 (here): CTA tiles of P = 128 lattice points, in
//      panels of 32 variables: the panel's conditional means
//      u_v - sum_{t < v0} L_vt y_t are a register-tiled contraction of the
//      panel's rows of L with the stored y history (smem-staged chunks of 32
//      variables), then one thread per point runs the panel's variables in
//      order (the in-panel terms, Phi, the running product, Phi^{-1} of the
//      lattice-weighted probability) and appends its y values to the history.
//      Mixed: the same recursion with the contraction on the tensor cores
//      (full_tc.cu);
//   5. per-block sums of the point products, added per shift in a fixed order.
#include <climits>
#include <tuple>
#include <map>
#include <mutex>

#include "cov.cuh"
#include "vk_internal.h"

namespace vk {
namespace {

constexpr int kCholB = 32;   // Cholesky block
constexpr int kFullP = 128;  // lattice points per CTA (one per thread in the sequential part)
constexpr int kFullKC = 32;  // history chunk of the contraction

__global__ void full_cov_kernel(const double* __restrict__ sites, int D, CovParams cv, double* __restrict__ A) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (r >= D || c > r) return;
    const double h = site_dist(cv, __dsub_rn(sites[2 * r], sites[2 * c]), __dsub_rn(sites[2 * r + 1], sites[2 * c + 1]));
    double v = cov_fn(cv.cov_kind, cv.variance, cv.range, cv.nu, h);
    if (c == r) v += cv.nugget;
    A[(int64_t)r * D + c] = v;
}

// Entry e of a packed lower triangle (e = r (r + 1) / 2 + c, c <= r).
__device__ __forceinline__ void tri_rc(int e, int& r, int& c) {
    r = (int)((sqrtf((float)(8 * e + 1)) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    while (r * (r + 1) / 2 > e) --r;
    c = e - r * (r + 1) / 2;
}

// 1/sqrt(s) for a positive normal double: the hardware approximation
// (rsqrt.approx.f64, about 2^-22 relative) and two Newton-Raphson steps
// y <- y + y (1 - s y^2) / 2, each squaring the relative error -- inline (a
// library call would spill the caller's registers around it).
__device__ __forceinline__ double rsqrt_nr(double s) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(s));
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double r = fma(-(s * y), y, 1.0);
        y = fma(0.5 * y, r, y);
    }
    return y;
}

// The pairs (row, column) of a packed lower triangle, in packed order: the
// pairs of an n x n triangle are the table's first n (n + 1) / 2 entries.
__device__ __forceinline__ void pair_table(unsigned short* tab) {
    for (int e = threadIdx.x; e < kCholB * (kCholB - 1) / 2; e += blockDim.x) {
        int r, c;
        tri_rc(e, r, c);
        tab[e] = (unsigned short)((r << 8) | c);
    }
}

// Factor the b x b block T in shared memory, all threads of the CTA,
// right-looking: at step j the column below the pivot is divided by it (FAST:
// multiplied by its reciprocal square root, a shorter dependent chain on
// GB300's 1/64-rate FP64 unit than a square root and a division), then the
// packed trailing triangle takes one fma per entry, spread over the threads
// through the pair table.  (Taking the next pivot's root inside the trailing
// update, by the thread that updates that entry, was slower: 31 against 26 us
// a block.)  Returns the first non-positive pivot, or -1.
template <bool FAST>
__device__ int factor_block(double (*T)[kCholB + 1], const unsigned short* tab, int b) {
    const int tid = threadIdx.x;
    for (int j = 0; j < b; ++j) {
        const double s = T[j][j];
        if (!(s > 0.0)) return j;  // block-uniform
        double piv = 0.0;
        if (tid < 32) {  // the pivot and its column: one warp (the others would only repeat it)
            if constexpr (FAST) {
                const double rs = rsqrt_nr(s);
                piv = s * rs;
                if (tid < b - 1 - j) T[j + 1 + tid][j] = T[j + 1 + tid][j] * rs;
            } else {
                piv = sqrt(s);
                if (tid < b - 1 - j) T[j + 1 + tid][j] = T[j + 1 + tid][j] / piv;
            }
        }
        __syncthreads();
        if (tid == 0) T[j][j] = piv;
        const int n = b - 1 - j;
        for (int e = tid; e < n * (n + 1) / 2; e += blockDim.x) {
            const unsigned t = tab[e];
            const int r = j + 1 + (int)(t >> 8), cc = j + 1 + (int)(t & 255u);
            T[r][cc] = fma(-T[r][j], T[cc][j], T[r][cc]);
        }
        __syncthreads();
    }
    return -1;
}

// The diagonal block at k0, 512 threads (one trailing entry a thread at the
// first pivots, so thread 0 holds only the next pivot).  FP64 path: each entry of the factor
// receives its terms in ascending order with fma and the pivot division last;
// FAST (mixed path): pivots from reciprocal square roots.  (Tried for the
// mixed path and slower: one warp holding the block in registers and
// shuffling the columns, 49 against 26 us a block, all its FP64 work on one
// SMSP; the factor repeated by every CTA of the row solve, 70 us a block
// column, the SMs' FP64 units shared with the trailing update.)
// upd (mixed path, k0 >= 32): the block first takes the update by the block
// column before it (rows k0 .. k0 + 31 of that solved panel, fma in ascending
// column order), which the tensor-core update of that column leaves out, so
// that this factor waits only for the row solve of the column before and not
// for the update of its whole first tile column.
template <bool FAST>
__global__ void __launch_bounds__(512) chol_diag_kernel(double* __restrict__ A, int D, int k0,
                                                        int* __restrict__ bad, int upd) {
    __shared__ double T[kCholB][kCholB + 1];
    __shared__ double P[kCholB][kCholB + 1];
    __shared__ unsigned short tab[kCholB * (kCholB - 1) / 2];
    const int b = min(kCholB, D - k0);
    for (int e = threadIdx.x; e < b * (b + 1) / 2; e += blockDim.x) {
        int r, c;
        tri_rc(e, r, c);
        T[r][c] = A[(int64_t)(k0 + r) * D + k0 + c];
    }
    if (upd)
        for (int x = threadIdx.x; x < b * kCholB; x += blockDim.x) {
            const int r = x / kCholB, t = x % kCholB;
            P[r][t] = A[(int64_t)(k0 + r) * D + k0 - kCholB + t];
        }
    pair_table(tab);
    __syncthreads();
    if (upd) {
        for (int e = threadIdx.x; e < b * (b + 1) / 2; e += blockDim.x) {
            int r, c;
            tri_rc(e, r, c);
            double acc = T[r][c];
#pragma unroll
            for (int t = 0; t < kCholB; ++t) acc = fma(-P[r][t], P[c][t], acc);
            T[r][c] = acc;
        }
        __syncthreads();
    }
    const int fail = factor_block<FAST>(T, tab, b);
    if (fail >= 0) {
        if (threadIdx.x == 0) atomicMin(bad, k0 + fail);
        return;
    }
    for (int e = threadIdx.x; e < b * (b + 1) / 2; e += blockDim.x) {
        int r, c;
        tri_rc(e, r, c);
        A[(int64_t)(k0 + r) * D + k0 + c] = T[r][c];
    }
}

// Rows r >= k0 + 32 of the block column: x L_kk^T = a by forward
// substitution, one thread per row, blockDim.x (8 to 32) rows per CTA.  The
// solve is right-looking: once x_j is known it goes into every later
// accumulator, so each x_k still receives its terms in ascending j with fma
// (bit for bit the row-by-row definition's sums).  Each entry divides by its
// pivot (the definition's operation: a reciprocal would change the factor's
// last bits, and with them which exactly singular block is reported).
__global__ void chol_trsm_kernel(double* __restrict__ A, int D, int k0) {
    __shared__ double Lk[kCholB][kCholB + 1];
    // the diagonal block, a row per thread and pass with its 32 loads issued
    // together (a CTA has as few as 8 threads: a load loop would wait on L2
    // 128 times in sequence)
    for (int r = threadIdx.x; r < kCholB; r += blockDim.x) {
        const double* src = A + (int64_t)(k0 + r) * D + k0;
        double v[kCholB];
#pragma unroll
        for (int c = 0; c < kCholB; ++c) v[c] = (c <= r) ? src[c] : 0.0;
#pragma unroll
        for (int c = 0; c < kCholB; ++c) Lk[r][c] = v[c];
    }
    __syncthreads();
    const int r = k0 + kCholB + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double* row = A + (int64_t)r * D + k0;
    double x[kCholB];
#pragma unroll
    for (int j = 0; j < kCholB; ++j) x[j] = row[j];
#pragma unroll
    for (int j = 0; j < kCholB; ++j) {
        x[j] = x[j] / Lk[j][j];
#pragma unroll
        for (int k = j + 1; k < kCholB; ++k) x[k] = fma(-x[j], Lk[k][j], x[k]);
    }
#pragma unroll
    for (int j = 0; j < kCholB; ++j) row[j] = x[j];
}

// Rows r >= k0 + 32 of the block column for the mixed path, whose trailing
// update runs on the tensor cores (chol_tc.cu): one warp per row, lane j
// holding x_j.  Step j: lane j multiplies its accumulator by the pivot's
// reciprocal, the warp shuffles x_j out and lanes k > j take fma(-x_j, L_kj, .)
// -- two FP64 warp instructions a column instead of a thread's 528 fma and 32
// divisions (GB300's FP64 unit costs the same per warp instruction however
// many lanes it carries).  The solved row then goes out for the tensor cores:
// its exponent e (|L_rt| 2^-e < 1) and the balanced base-256 digits s_0 ..
// s_6 of round(L_rt 2^(56 - e)), bf16, in the operand layout of its 8-row
// group (rel = r - k0 - 32).
constexpr int kSolveWarps = 4;
__global__ void __launch_bounds__(kSolveWarps * 32) chol_trsm_slice_kernel(double* __restrict__ A, int D, int k0,
                                                                           unsigned char* __restrict__ sl,
                                                                           int* __restrict__ ex) {
    __shared__ double T[kCholB][kCholB + 1];
    __shared__ double rinv[kCholB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {  // the factored diagonal block: 8 loads a thread, issued together
        const int r = tid >> 2, c0 = (tid & 3) * 8;
        const double* src = A + (int64_t)(k0 + r) * D + k0 + c0;
        double v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = (c0 + c <= r) ? src[c] : 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) T[r][c0 + c] = v[c];
    }
    __syncthreads();
    if (tid < kCholB) rinv[tid] = 1.0 / T[tid][tid];
    __syncthreads();
    const int r = k0 + kCholB + blockIdx.x * kSolveWarps + warp;
    if (r >= D) return;  // warp-uniform
    double* row = A + (int64_t)r * D + k0;
    double acc = row[lane];
#pragma unroll
    for (int j = 0; j < kCholB; ++j) {
        if (lane == j) acc *= rinv[j];
        const double xj = __shfl_sync(0xffffffffu, acc, j);
        if (lane > j) acc = fma(-xj, T[lane][j], acc);
    }
    row[lane] = acc;
    // exponent of the row's largest entry (zeros and subnormals: the rows of
    // a zero block column, left at e = 0)
    const unsigned E = (unsigned)((__double_as_longlong(acc) >> 52) & 0x7FF);
    const unsigned Emax = __reduce_max_sync(0xffffffffu, E);
    const int e = (Emax == 0) ? 0 : max((int)Emax - 1022, -900);
    const double sc = __hiloint2double((56 - e + 1023) << 20, 0);  // 2^(56 - e)
    const int rel = r - k0 - kCholB;
    if (lane == 0) ex[rel] = e;
    long long X = __double2ll_rn(acc * sc);  // |X| <= 2^56
    int d[kCholSlices];
#pragma unroll
    for (int i = kCholSlices - 1; i >= 1; --i) {
        d[i] = (int)((X + 128) & 255) - 128;
        X = (X - d[i]) >> 8;
    }
    d[0] = (int)X;  // |d_0| <= 256
    unsigned char* grp = sl + (size_t)(rel >> 3) * kCholSliceGroupBytes + (rel & 7) * 16 + (lane >> 3) * 128 +
                         (lane & 7) * 2;
#pragma unroll
    for (int i = 0; i < kCholSlices; ++i) {
        const uint32_t h = __float_as_uint((float)d[i]) >> 16;  // exact in bf16
        const uint32_t hn = __shfl_down_sync(0xffffffffu, h, 1);
        if (!(lane & 1)) *reinterpret_cast<uint32_t*>(grp + i * 512) = h | (hn << 16);
    }
}

// Trailing update of the lower triangle below block column k0, 256 threads.
// part 0: the first tile column (the next block column, on the factor's
// critical path) in chunks of 8 rows x 32 columns, one entry per thread, so
// that it spreads over 4x more SMs; part 1: the 32 x 32 tiles (tile rows >=
// tile columns) of the tile columns after it, 4 entries per thread.
__global__ void chol_update_kernel(double* __restrict__ A, int D, int k0, int part) {
    __shared__ double Lr[kCholB][kCholB + 1], Lc[kCholB][kCholB + 1];
    const int base = k0 + kCholB;
    // rows r0 .. r0 + rows - 1 against the columns c0 .. c0 + 31
    int r0, c0, rows;
    if (part == 0) {
        r0 = base + blockIdx.x * 8;
        c0 = base;
        rows = 8;
    } else {  // tile pair (tr, tc), tc <= tr, from the linear block index
        int tr, tc;
        tri_rc(blockIdx.x, tr, tc);
        r0 = base + (tr + 1) * kCholB;
        c0 = base + (tc + 1) * kCholB;
        rows = kCholB;
    }
    for (int x = threadIdx.x; x < kCholB * kCholB; x += blockDim.x) {
        const int i = x / kCholB, t = x % kCholB;
        if (i < rows) Lr[i][t] = (r0 + i < D) ? A[(int64_t)(r0 + i) * D + k0 + t] : 0.0;
        Lc[i][t] = (c0 + i < D) ? A[(int64_t)(c0 + i) * D + k0 + t] : 0.0;
    }
    __syncthreads();
    const int j = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < rows; i += blockDim.x >> 5) {
        const int r = r0 + i, c = c0 + j;
        if (r >= D || c > r) continue;
        double acc = A[(int64_t)r * D + c];
#pragma unroll
        for (int t = 0; t < kCholB; ++t) acc = fma(-Lr[i][t], Lc[j][t], acc);
        A[(int64_t)r * D + c] = acc;
    }
}

// Scaled tables: Ls[v][t] = L_vt / L_vv (t < v), us[v] = u_v / L_vv.
template <class T>
__global__ void full_tables_kernel(const double* __restrict__ A, const double* __restrict__ u, int D,
                                   T* __restrict__ Ls, T* __restrict__ us) {
    const int v = blockIdx.y;
    const double rd = 1.0 / A[(int64_t)v * D + v];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < D; t += gridDim.x * blockDim.x)
        Ls[(int64_t)v * D + t] = (t < v) ? (T)(A[(int64_t)v * D + t] * rd) : (T)0;
    if (blockIdx.x == 0 && threadIdx.x == 0) us[v] = (T)(u[v] * rd);
}

// ---- the recursion ----------------------------------------------------------

template <class T>
struct FullTraits;
template <>
struct FullTraits<double> {
    static constexpr int B = 32, TJ = 4, TP = 8;  // panel width; per-thread tile (variables x points)
};

struct FullArgs {
    int D;
    int64_t N;
    int S;
    int blocks_per_shift;
    const uint32_t* g;     // lattice vector, D - 1 entries
    const double* delta;   // S x dim shifts
    int dim;               // row stride of delta
};

// e = Phi(z), ec = 1 - e.
__device__ __forceinline__ void full_phi(double z, double& e, double& ec) {
    const double t = normcdf(-fabs(z));
    e = (z < 0.0) ? t : 1.0 - t;
    ec = (z < 0.0) ? 1.0 - t : t;
}

// y = Phi^{-1}(w e) at lattice coordinate v of point k of shift s.
__device__ __forceinline__ double full_y(const FullArgs& a, int s, uint32_t k, int v, double e, double ec) {
    const uint64_t rr = ((uint64_t)k * (uint64_t)a.g[v]) % (uint64_t)a.N;
    double x = __dadd_rn((double)rr / (double)a.N, a.delta[(int64_t)s * a.dim + v]);
    if (x >= 1.0) x -= 1.0;
    const double am = fabs(__dsub_rn(__dmul_rn(2.0, x), 1.0));
    const double w = __dsub_rn(1.0, am);
    const double p = __dmul_rn(w, e), q = __dadd_rn(am, __dmul_rn(w, ec));
    const double lo = 9.3326361850321887899e-302;  // 2^-1000
    const double pc = fmax(p, lo), qc = fmax(q, lo);
    return (pc <= qc) ? normcdfinv(pc) : -normcdfinv(qc);
}

template <class T>
__global__ void __launch_bounds__(kFullP) full_genz_kernel(const T* __restrict__ Ls, const T* __restrict__ us,
                                                           FullArgs a, T* __restrict__ Y,
                                                           double* __restrict__ part) {
    constexpr int B = FullTraits<T>::B, TJ = FullTraits<T>::TJ, TP = FullTraits<T>::TP;
    constexpr int P = kFullP, KC = kFullKC;
    static_assert((B / TJ) * (P / TP) == kFullP, "thread tile");
    extern __shared__ __align__(16) unsigned char full_smem[];
    T* Ych = (T*)full_smem;        // [KC][P]
    T* Lch = Ych + KC * P;         // [B][KC + 1]
    T* Zs = Lch + B * (KC + 1);    // [B][P]: conditional means, then the panel's y
    T* Lp = Zs + B * P;            // [B][B + 1]: the panel's own triangle
    __shared__ double red[kFullP / 32];
    const int tid = threadIdx.x, D = a.D;
    const int s = blockIdx.x / a.blocks_per_shift;
    const int64_t k64 = (int64_t)(blockIdx.x % a.blocks_per_shift) * P + tid;
    const bool valid = k64 < a.N;
    const uint32_t k = (uint32_t)(valid ? k64 : a.N - 1);
    T* Yb = Y + (int64_t)blockIdx.x * D * P;  // this tile's y history [D][P]
    const int tj = tid / (P / TP), tp = tid % (P / TP);  // thread tile (variables tj*TJ.., points tp*TP..)
    double f = 1.0;
    for (int v0 = 0; v0 < D; v0 += B) {
        const int nb = min(B, D - v0);
        // the panel's triangle
        for (int x = tid; x < B * B; x += P) {
            const int j = x / B, i = x % B;
            Lp[j * (B + 1) + i] = (j < nb && i < j) ? Ls[(int64_t)(v0 + j) * D + v0 + i] : (T)0;
        }
        // conditional means from the history: Zs[j][p] = us_v - sum_{t < v0} Ls[v][t] y_t[p]
        T acc[TJ][TP];
#pragma unroll
        for (int i = 0; i < TJ; ++i)
#pragma unroll
            for (int q = 0; q < TP; ++q) acc[i][q] = (T)0;
        for (int t0 = 0; t0 < v0; t0 += KC) {
            __syncthreads();  // previous chunk consumed
            for (int x = tid; x < KC * P; x += P) {
                const int tt = x / P, p = x % P;
                Ych[x] = Yb[(int64_t)(t0 + tt) * P + p];
            }
            for (int x = tid; x < B * KC; x += P) {
                const int j = x / KC, tt = x % KC;
                Lch[j * (KC + 1) + tt] = (j < nb) ? Ls[(int64_t)(v0 + j) * D + t0 + tt] : (T)0;
            }
            __syncthreads();
#pragma unroll 4
            for (int tt = 0; tt < KC; ++tt) {
                T lv[TJ], yv[TP];
#pragma unroll
                for (int i = 0; i < TJ; ++i) lv[i] = Lch[(tj * TJ + i) * (KC + 1) + tt];
#pragma unroll
                for (int q = 0; q < TP; ++q) yv[q] = Ych[tt * P + tp * TP + q];
#pragma unroll
                for (int i = 0; i < TJ; ++i)
#pragma unroll
                    for (int q = 0; q < TP; ++q) acc[i][q] = fma(lv[i], yv[q], acc[i][q]);
            }
        }
#pragma unroll
        for (int i = 0; i < TJ; ++i) {
            const int j = tj * TJ + i;
            const T uv = (j < nb) ? us[v0 + j] : (T)0;
#pragma unroll
            for (int q = 0; q < TP; ++q) Zs[j * P + tp * TP + q] = uv - acc[i][q];
        }
        __syncthreads();
        // the panel's variables in order, one thread per point
        const int p = tid;
        for (int j = 0; j < nb; ++j) {
            const int v = v0 + j;
            T z = Zs[j * P + p];
            for (int i = 0; i < j; ++i) z = fma(-Lp[j * (B + 1) + i], Zs[i * P + p], z);
            T e, ec;
            full_phi(z, e, ec);
            f *= (double)e;
            if (v < D - 1) Zs[j * P + p] = full_y(a, s, k, v, e, ec);
        }
        for (int j = 0; j < nb; ++j)
            if (v0 + j < D - 1) Yb[(int64_t)(v0 + j) * P + p] = Zs[j * P + p];
        __syncthreads();  // Zs and Lp reused by the next panel
    }
    // tile sum of the point products, fixed order
    double v = valid ? f : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kFullP / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

template <class T>
size_t full_smem_bytes() {
    constexpr int B = FullTraits<T>::B;
    return sizeof(T) * ((size_t)kFullKC * kFullP + (size_t)B * (kFullKC + 1) + (size_t)B * kFullP +
                        (size_t)B * (B + 1));
}

template <class T>
cudaError_t launch_full_genz_t(const double* A, const double* u, const FullArgs& a, void* Ls, void* us, void* Y,
                               double* part, cudaEvent_t ev_begin, cudaEvent_t ev_end, cudaStream_t st) {
    const int D = a.D;
    full_tables_kernel<T><<<dim3((D + 255) / 256 > 8 ? 8 : (D + 255) / 256, D), 256, 0, st>>>(A, u, D, (T*)Ls, (T*)us);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = full_smem_bytes<T>();
    static std::mutex mu;
    static std::map<int, bool> attr;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr[dev]) {
            e = cudaFuncSetAttribute(full_genz_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
    }
    const int blocks = a.S * a.blocks_per_shift;
    if (ev_begin && (e = cudaEventRecord(ev_begin, st)) != cudaSuccess) return e;
    full_genz_kernel<T><<<blocks, kFullP, smem, st>>>((const T*)Ls, (const T*)us, a, (T*)Y, part);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev_end) e = cudaEventRecord(ev_end, st);
    return e;
}

}  // namespace

// Rows per CTA of the row solve: 32 while that still gives every SM a CTA,
// else fewer (down to 8), so the solve of a block column uses as many of the
// SMs' FP64 units as its rows allow.
int trsm_rows_per_cta(int64_t rows, int64_t sms) {
    return rows >= 32 * sms ? 32 : rows >= 16 * sms ? 16 : 8;
}

// Blocked Cholesky with a one-block lookahead on two streams.  The caller's
// stream st carries the critical path: update of block column k by step k-1,
// then its diagonal factor and the rows below it; a second stream applies the
// rest of step k's trailing update meanwhile.  Every entry still receives the
// steps' terms in ascending order: the rest of step k-1 finishes before the
// first-column update of step k, and each stream keeps its own order.
size_t chol_tc_scratch_bytes(int64_t D) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return 2 * (al(chol_tc_slice_bytes(D)) + al(sizeof(int) * (size_t)(D + 128)));
}

// The side streams and events of one factorization (created per call, so
// that concurrent calls on other streams share nothing).
struct CholStreams {
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_rest[2] = {nullptr, nullptr}, ev_p0[2] = {nullptr, nullptr};
    cudaError_t create(bool tc) {
        cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev_rest[i], cudaEventDisableTiming);
        if (tc) {
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&side2, cudaStreamNonBlocking);
            for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev_p0[i], cudaEventDisableTiming);
        }
        return e;
    }
    ~CholStreams() {  // work still queued completes first (the runtime defers the release)
        if (ev_panel) cudaEventDestroy(ev_panel);
        for (int i = 0; i < 2; ++i) {
            if (ev_rest[i]) cudaEventDestroy(ev_rest[i]);
            if (ev_p0[i]) cudaEventDestroy(ev_p0[i]);
        }
        if (side) cudaStreamDestroy(side);
        if (side2) cudaStreamDestroy(side2);
    }
};

// The blocked factor of the covariance in A (see launch_cov_chol), queued on st.
cudaError_t enqueue_chol(double* A, int64_t D, int* bad, cudaStream_t st, void* tc_scratch, int* timeout,
                         uint64_t wait_ns, int64_t sms, CholStreams& cs) {
    cudaError_t e = cudaSuccess;
    const int64_t nblk = (D + kCholB - 1) / kCholB;
    if (nblk <= 2 || e != cudaSuccess) {  // nothing to overlap
        for (int64_t k0 = 0; k0 < D && e == cudaSuccess; k0 += kCholB) {
            chol_diag_kernel<false><<<1, 512, 0, st>>>(A, (int)D, (int)k0, bad, 0);
            const int64_t rows = D - k0 - kCholB;
            if (rows > 0) {
                const int rb = trsm_rows_per_cta(rows, sms);
                chol_trsm_kernel<<<(unsigned)((rows + rb - 1) / rb), rb, 0, st>>>(A, (int)D, (int)k0);
                chol_update_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(A, (int)D, (int)k0, 0);
            }
            e = cudaGetLastError();
        }
        return e;
    }
    // tensor-core updates: slice buffers and exponents, one pair per parity of
    // the block column (the side stream's update of column k still reads its
    // slices while the row solve of column k + 1 writes the other pair)
    const bool tc = tc_scratch != nullptr;
    unsigned char* slb[2] = {nullptr, nullptr};
    int* exb[2] = {nullptr, nullptr};
    if (tc) {
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        char* q = (char*)tc_scratch;
        for (int i = 0; i < 2; ++i) {
            slb[i] = (unsigned char*)q;
            q += al(chol_tc_slice_bytes(D));
            exb[i] = (int*)q;
            q += al(sizeof(int) * (size_t)(D + 128));
        }
    }
    cudaStream_t side = cs.side, side2 = cs.side2;
    cudaEvent_t ev_panel = cs.ev_panel;
    cudaEvent_t* ev_rest = cs.ev_rest;
    cudaEvent_t* ev_p0 = cs.ev_p0;
    if (tc && e == cudaSuccess) {
        // Critical stream: row solve of column k, then the factor of block
        // k + 1 (which applies column k's update to its own block), then the
        // solve of column k + 1 once the tensor-core update of column k + 1's
        // other rows (side2) is in.  side: the rest of the trailing update.
        chol_diag_kernel<true><<<1, 512, 0, st>>>(A, (int)D, 0, bad, 0);
        for (int64_t k = 0; k < nblk && e == cudaSuccess; ++k) {
            const int64_t k0 = k * kCholB, rows = D - k0 - kCholB;
            if (rows <= 0) break;
            chol_trsm_slice_kernel<<<(unsigned)((rows + kSolveWarps - 1) / kSolveWarps), kSolveWarps * 32, 0, st>>>(
                A, (int)D, (int)k0, slb[k & 1], exb[k & 1]);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(ev_panel, st);
            const int64_t tiles = (rows + kCholB - 1) / kCholB;
            if (tiles > 1) {
                if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_panel, 0);
                if (e == cudaSuccess)
                    e = launch_chol_update_tc(slb[k & 1], exb[k & 1], A, D, k0 + kCholB, 1, timeout, wait_ns, side);
                if (e == cudaSuccess) e = cudaEventRecord(ev_rest[k & 1], side);
            }
            // column k + 1 below its diagonal block: after the solve of k and
            // the rest of step k - 1 (launched whenever this step has rows)
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side2, ev_panel, 0);
            if (k > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(side2, ev_rest[(k - 1) & 1], 0);
            if (e == cudaSuccess)
                e = launch_chol_update_tc(slb[k & 1], exb[k & 1], A, D, k0 + kCholB, 0, timeout, wait_ns, side2);
            if (e == cudaSuccess) e = cudaEventRecord(ev_p0[k & 1], side2);
            // block k + 1, which the rest of step k - 1 has updated
            if (k > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_rest[(k - 1) & 1], 0);
            if (e == cudaSuccess) {
                chol_diag_kernel<true><<<1, 512, 0, st>>>(A, (int)D, (int)(k0 + kCholB), bad, 1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_p0[k & 1], 0);
        }
    }
    for (int64_t k = 0; !tc && k < nblk && e == cudaSuccess; ++k) {
        const int64_t k0 = k * kCholB, rows = D - k0 - kCholB;
        chol_diag_kernel<false><<<1, 512, 0, st>>>(A, (int)D, (int)k0, bad, 0);
        if (rows <= 0) {
            e = cudaGetLastError();
            break;
        }
        const int rb = trsm_rows_per_cta(rows, sms);
        chol_trsm_kernel<<<(unsigned)((rows + rb - 1) / rb), rb, 0, st>>>(A, (int)D, (int)k0);
        const int64_t tiles = (rows + kCholB - 1) / kCholB;
        if (tiles > 1) {  // the rest of step k on the side stream
            if (e == cudaSuccess) e = cudaEventRecord(ev_panel, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_panel, 0);
            if (e == cudaSuccess) {
                chol_update_kernel<<<(unsigned)(tiles * (tiles - 1) / 2), 256, 0, side>>>(A, (int)D, (int)k0, 1);
                e = cudaEventRecord(ev_rest[k & 1], side);
            }
        }
        // the first column of step k needs the rest of step k - 1
        if (k > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_rest[(k - 1) & 1], 0);
        if (e == cudaSuccess) {
            chol_update_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(A, (int)D, (int)k0, 0);
            e = cudaGetLastError();
        }
    }
    // the last rest update joins the caller's stream
    if (e == cudaSuccess) {
        const int64_t last = nblk - 2;  // the last step with a trailing matrix of more than one tile
        for (int64_t k = last; k >= 0; --k)
            if ((D - k * kCholB - kCholB + kCholB - 1) / kCholB > 1) {
                e = cudaStreamWaitEvent(st, ev_rest[k & 1], 0);
                break;
            }
    }
    return e;
}

// The mixed factor's few hundred small launches and stream waits per call
// are replayed from a CUDA graph captured once per (device, D, buffers):
// queued one by one, the host needs about as long per block column as the
// GPU.  The graph is captured on a private stream (after the tensor-core
// kernel's attributes are set, outside the capture) and launched on the
// caller's, which may be the legacy default stream; on a stream the caller
// is itself capturing, the factor is queued eagerly.
namespace {
struct CholGraphKey {
    int dev;
    int64_t D;
    const void *A, *bad, *scratch, *timeout;
    uint64_t wait_ns;
    bool operator<(const CholGraphKey& o) const {
        return std::tie(dev, D, A, bad, scratch, timeout, wait_ns) <
               std::tie(o.dev, o.D, o.A, o.bad, o.scratch, o.timeout, o.wait_ns);
    }
};
std::mutex g_chol_mu;
std::map<CholGraphKey, cudaGraphExec_t> g_chol_graphs;
constexpr size_t kMaxCholGraphs = 32;
}  // namespace

cudaError_t launch_cov_chol(const double* sites, int64_t D, const vecchia_cov& cov, double* A, int* bad,
                            cudaStream_t st, void* tc_scratch, int* timeout, uint64_t wait_ns) {
    if (D <= 0) return cudaSuccess;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    const int64_t sms = device_sm_count(dev);
    full_cov_kernel<<<dim3((unsigned)((D + 127) / 128), (unsigned)D), 128, 0, st>>>(sites, (int)D, cov_params(cov), A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool tc = tc_scratch != nullptr;
    const int64_t nblk = (D + kCholB - 1) / kCholB;
    bool graph = tc && nblk > 2;
    if (graph) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        graph = cudaStreamIsCapturing(st, &cst) == cudaSuccess && cst == cudaStreamCaptureStatusNone;
    }
    const CholGraphKey key{dev, D, A, bad, tc_scratch, timeout, wait_ns};
    if (graph) {
        std::lock_guard<std::mutex> lk(g_chol_mu);
        auto it = g_chol_graphs.find(key);
        if (it != g_chol_graphs.end()) return cudaGraphLaunch(it->second, st);
    }
    if (tc) {
        e = chol_tc_prepare();
        if (e != cudaSuccess) return e;
    }
    CholStreams cs;
    e = cs.create(tc);
    if (e != cudaSuccess) return e;
    if (!graph) return enqueue_chol(A, D, bad, st, tc_scratch, timeout, wait_ns, sms, cs);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;  // capture only: nothing runs on it
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t eq = enqueue_chol(A, D, bad, cap, tc_scratch, timeout, wait_ns, sms, cs);
        e = cudaStreamEndCapture(cap, &g);
        if (eq != cudaSuccess) e = eq;
    }
    if (cap) cudaStreamDestroy(cap);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {  // not capturable here: queue it eagerly
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        return enqueue_chol(A, D, bad, st, tc_scratch, timeout, wait_ns, sms, cs);
    }
    {
        std::lock_guard<std::mutex> lk(g_chol_mu);
        if (g_chol_graphs.size() >= kMaxCholGraphs) {
            for (auto& kv : g_chol_graphs) cudaGraphExecDestroy(kv.second);
            g_chol_graphs.clear();
        }
        g_chol_graphs[key] = exec;
    }
    return cudaGraphLaunch(exec, st);
}

int64_t full_genz_blocks_per_shift(int64_t N, bool mixed) {
    return mixed ? full_tc_blocks_per_shift(N) : (N + kFullP - 1) / kFullP;
}

// Scratch: the shared part (factor, lattice and shift tables, block sums,
// status words) followed by the precision's own tables and y history.
size_t full_genz_scratch_bytes(int64_t D, int64_t N, int S, bool mixed) {
    const int64_t bps = (N + kFullP - 1) / kFullP, nblk = full_genz_blocks_per_shift(N, mixed);
    const int64_t dim = D > 1 ? D - 1 : 1;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t shared = al(sizeof(double) * D * D) + al(sizeof(uint32_t) * dim * 2) + al(sizeof(double) * S * dim) +
                          al(sizeof(uint32_t) * S * dim) + al(sizeof(double) * S * nblk) + al(2 * sizeof(int)) +
                          al(sizeof(uint64_t) + 2 * sizeof(int64_t) + sizeof(int32_t));
    if (mixed) return shared + al(chol_tc_scratch_bytes(D)) + full_tc_scratch_bytes(D, N, S);
    return shared + al(sizeof(double) * D * D) + al(sizeof(double) * D) + al(sizeof(double) * (size_t)S * bps * D * kFullP);
}

cudaError_t launch_full_genz(const double* sites, const double* u, int64_t D, const vecchia_cov& cov, int64_t N,
                             int S, bool mixed, const uint32_t* g_host, const uint32_t* gfix_host,
                             uint64_t seed, void* scratch, double* part_host, int* bad_host, int* timeout_host,
                             uint64_t wait_ns, int withhold, cudaEvent_t ev_begin, cudaEvent_t ev_end,
                             cudaStream_t st) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int64_t bps = (N + kFullP - 1) / kFullP, nblk = full_genz_blocks_per_shift(N, mixed);
    const int64_t dim = D > 1 ? D - 1 : 1;
    char* p = (char*)scratch;
    double* A = (double*)p;
    p += al(sizeof(double) * D * D);
    uint32_t* gdev = (uint32_t*)p;
    p += al(sizeof(uint32_t) * dim * 2);
    double* delta = (double*)p;
    p += al(sizeof(double) * S * dim);
    uint32_t* dfix = (uint32_t*)p;
    p += al(sizeof(uint32_t) * S * dim);
    double* part = (double*)p;
    p += al(sizeof(double) * S * nblk);
    int* bad = (int*)p;  // bad[0]: first failing pivot; bad[1]: a device wait timed out
    p += al(2 * sizeof(int));
    char* small = p;  // seed, offset, S for the shift kernel
    p += al(sizeof(uint64_t) + 2 * sizeof(int64_t) + sizeof(int32_t));
    uint64_t* seed_d = (uint64_t*)small;
    int64_t* off_d = (int64_t*)(small + sizeof(uint64_t));
    int32_t* S_d = (int32_t*)(small + sizeof(uint64_t) + 2 * sizeof(int64_t));

    const int status_init[2] = {INT_MAX, 0};
    cudaError_t e = cudaMemcpyAsync(bad, status_init, sizeof(status_init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gdev, g_host, sizeof(uint32_t) * dim, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gdev + dim, gfix_host, sizeof(uint32_t) * dim, cudaMemcpyHostToDevice, st);
    const int64_t zero = 0;
    const int32_t S32 = S;
    if (e == cudaSuccess) e = cudaMemcpyAsync(seed_d, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(off_d, &zero, sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S_d, &S32, sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = launch_shifts(seed_d, S_d, off_d, 1, (int)dim, delta, dfix, st);
    if (e != cudaSuccess) return e;
    if (mixed) {  // the factor's trailing updates on the tensor cores
        e = launch_cov_chol(sites, D, cov, A, bad, st, p, bad + 1, wait_ns);
        p += al(chol_tc_scratch_bytes(D));
    } else {
        e = launch_cov_chol(sites, D, cov, A, bad, st);
    }
    if (e != cudaSuccess) return e;
    if (mixed) {
        e = launch_full_genz_tc(A, u, D, N, S, gdev + dim, dfix, (int)dim, p, part, bad + 1, wait_ns, withhold,
                                ev_begin, ev_end, st);
    } else {
        void* Ls = p;
        p += al(sizeof(double) * D * D);
        void* us = p;
        p += al(sizeof(double) * D);
        void* Y = p;
        FullArgs fa;
        fa.D = (int)D;
        fa.N = N;
        fa.S = S;
        fa.blocks_per_shift = (int)bps;
        fa.g = gdev;
        fa.delta = delta;
        fa.dim = (int)dim;
        e = launch_full_genz_t<double>(A, u, fa, Ls, us, Y, part, ev_begin, ev_end, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(part_host, part, sizeof(double) * S * nblk, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(timeout_host, bad + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    return e;
}

}  // namespace vk
