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

// The diagonal block at k0 (128 threads): right-looking; at step j the column
// below the pivot is divided by it, then the packed trailing triangle takes one
// fma per entry, spread over the threads through a table of (row, column)
// pairs in packed order (the pairs of an n x n triangle are the table's first
// n (n + 1) / 2 entries).
__global__ void __launch_bounds__(128) chol_diag_kernel(double* __restrict__ A, int D, int k0,
                                                        int* __restrict__ bad) {
    __shared__ double T[kCholB][kCholB + 1];
    __shared__ unsigned short tab[kCholB * (kCholB - 1) / 2];
    const int tid = threadIdx.x;
    const int b = min(kCholB, D - k0);
    for (int e = tid; e < b * (b + 1) / 2; e += blockDim.x) {
        int r, c;
        tri_rc(e, r, c);
        T[r][c] = A[(int64_t)(k0 + r) * D + k0 + c];
    }
    for (int e = tid; e < kCholB * (kCholB - 1) / 2; e += blockDim.x) {
        int r, c;
        tri_rc(e, r, c);
        tab[e] = (unsigned short)((r << 8) | c);
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        const double s = T[j][j];
        if (!(s > 0.0)) {  // block-uniform
            if (tid == 0) atomicMin(bad, k0 + j);
            return;
        }
        const double piv = sqrt(s);
        if (tid < b - 1 - j) T[j + 1 + tid][j] = T[j + 1 + tid][j] / piv;
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
    for (int e = tid; e < b * (b + 1) / 2; e += blockDim.x) {
        int r, c;
        tri_rc(e, r, c);
        A[(int64_t)(k0 + r) * D + k0 + c] = T[r][c];
    }
}

// Rows r >= k0 + 32 of the block column: x L_kk^T = a by forward
// substitution, one thread per row.  Each entry divides by its pivot (the
// row-by-row definition's operation: a reciprocal would save FP64 work but
// change the factor's last bits, and with them which exactly singular
// block is reported).
__global__ void chol_trsm_kernel(double* __restrict__ A, int D, int k0) {
    __shared__ double Lk[kCholB][kCholB + 1];
    for (int x = threadIdx.x; x < kCholB * kCholB; x += blockDim.x) {
        const int r = x / kCholB, c = x % kCholB;
        Lk[r][c] = (c <= r) ? A[(int64_t)(k0 + r) * D + k0 + c] : 0.0;
    }
    __syncthreads();
    const int r = k0 + kCholB + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double* row = A + (int64_t)r * D + k0;
    double x[kCholB];
#pragma unroll
    for (int j = 0; j < kCholB; ++j) {
        double acc = row[j];
#pragma unroll
        for (int i = 0; i < j; ++i) acc = fma(-x[i], Lk[j][i], acc);
        x[j] = acc / Lk[j][j];
    }
#pragma unroll
    for (int j = 0; j < kCholB; ++j) row[j] = x[j];
}

// Trailing update of the lower triangle below block column k0: 32 x 32 tiles
// (tile rows >= tile columns), 256 threads, 4 entries each.  part 0: the first
// tile column (the next block column), one CTA per tile row; part 1: the tile
// columns after it.
__global__ void chol_update_kernel(double* __restrict__ A, int D, int k0, int part) {
    __shared__ double Lr[kCholB][kCholB + 1], Lc[kCholB][kCholB + 1];
    const int base = k0 + kCholB;
    // tile pair (tr, tc), tc <= tr, from the linear block index
    int tr, tc;
    if (part == 0) {
        tr = blockIdx.x;
        tc = 0;
    } else {
        tri_rc(blockIdx.x, tr, tc);
        ++tr;
        ++tc;
    }
    const int r0 = base + tr * kCholB, c0 = base + tc * kCholB;
    for (int x = threadIdx.x; x < kCholB * kCholB; x += blockDim.x) {
        const int i = x / kCholB, t = x % kCholB;
        Lr[i][t] = (r0 + i < D) ? A[(int64_t)(r0 + i) * D + k0 + t] : 0.0;
        Lc[i][t] = (c0 + i < D) ? A[(int64_t)(c0 + i) * D + k0 + t] : 0.0;
    }
    __syncthreads();
    const int j = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < kCholB; i += blockDim.x >> 5) {
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

// Blocked Cholesky with a one-block lookahead on two streams.  The caller's
// stream st carries the critical path: update of block column k by step k-1,
// then its diagonal factor and the rows below it; a second stream applies the
// rest of step k's trailing update meanwhile.  Every entry still receives the
// steps' terms in ascending order: the rest of step k-1 finishes before the
// first-column update of step k, and each stream keeps its own order.
cudaError_t launch_cov_chol(const double* sites, int64_t D, const vecchia_cov& cov, double* A, int* bad,
                            cudaStream_t st) {
    if (D <= 0) return cudaSuccess;
    full_cov_kernel<<<dim3((unsigned)((D + 127) / 128), (unsigned)D), 128, 0, st>>>(sites, (int)D, cov_params(cov), A);
    cudaError_t e = cudaGetLastError();
    const int64_t nblk = (D + kCholB - 1) / kCholB;
    if (nblk <= 2 || e != cudaSuccess) {  // nothing to overlap
        for (int64_t k0 = 0; k0 < D && e == cudaSuccess; k0 += kCholB) {
            chol_diag_kernel<<<1, 128, 0, st>>>(A, (int)D, (int)k0, bad);
            const int64_t rows = D - k0 - kCholB;
            if (rows > 0) {
                chol_trsm_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(A, (int)D, (int)k0);
                chol_update_kernel<<<1, 256, 0, st>>>(A, (int)D, (int)k0, 0);
            }
            e = cudaGetLastError();
        }
        return e;
    }
    cudaStream_t side = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_rest[2] = {nullptr, nullptr};
    e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_rest[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_rest[1], cudaEventDisableTiming);
    for (int64_t k = 0; k < nblk && e == cudaSuccess; ++k) {
        const int64_t k0 = k * kCholB, rows = D - k0 - kCholB;
        chol_diag_kernel<<<1, 128, 0, st>>>(A, (int)D, (int)k0, bad);
        if (rows <= 0) {
            e = cudaGetLastError();
            break;
        }
        chol_trsm_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(A, (int)D, (int)k0);
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
            chol_update_kernel<<<(unsigned)tiles, 256, 0, st>>>(A, (int)D, (int)k0, 0);
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
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_rest[0]) cudaEventDestroy(ev_rest[0]);
    if (ev_rest[1]) cudaEventDestroy(ev_rest[1]);
    if (side) cudaStreamDestroy(side);
    return e;
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
    if (mixed) return shared + full_tc_scratch_bytes(D, N, S);
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
    e = launch_cov_chol(sites, D, cov, A, bad, st);
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
