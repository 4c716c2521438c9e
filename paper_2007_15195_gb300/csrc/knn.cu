// knn.cu -- conditioning sets N(i): the min(m, i) nearest previously ordered
// sites of every ordered site i (Sec. 2.1; Eq. vecchia-pdf / vecchia-cdf use
// |N_i| = min(m, i-1) in 1-based indexing).
//
// Integer work throughout, so the result is exact and reproducible:
//   - quantise: q = floor((x - xmin) * c), c = 2^30 / max extent (FP64, no
//     contraction), giving coordinates in [0, 2^30];
//   - key of a candidate j for site i: (squared quantised distance, j), so
//     distance ties go to the smaller index;
//   - bucket the sites into a (G+1) x (G+1) grid of square cells of side
//     2^(30 - log2 G) by a counting sort;
//   - one warp per site visits rings of cells of growing Chebyshev radius r
//     around the site's cell, keeping the best q keys among sites j < i in a
//     warp-wide sorted list; after ring r every unvisited site is at least
//     r*cell + 1 away in one coordinate, so the search stops once the q-th
//     best squared distance is below (r*cell + 1)^2;
//   - sites with a small index are searched by brute force over j < i.
#include <climits>
#include <map>
#include <mutex>

#include "vk_internal.h"

namespace vk {
namespace {

constexpr int kBruteLimit = 512;

struct Grid {
    double xmin, ymin, c;
    int shift;  // cell = q >> shift
    int G;      // cells per axis minus one (q = 2^30 lands in cell G)
    int zero;   // all sites equal: every coordinate quantises to 0
};

int grid_bits(int64_t D) {
    int k = 0;
    while (k < 10 && (int64_t)(2 << k) * (2 << k) <= D / 2) ++k;  // (2^(k+1))^2 <= D/2
    return k;
}

// Order-preserving integer image of a double (-0 taken as +0, as the
// comparison x < y treats them): integer compares instead of FP64 ones, which
// GB300 runs at 1/64 of its FP32 rate.
__device__ __forceinline__ unsigned long long ord_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x == 0.0 ? 0.0 : x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double ord_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k));
}
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Bounding box of the sites (one CTA): minima of the keys of x, y and of
// their complements (the maxima), warp shuffles then one pass over the warps.
__global__ void bbox_kernel(const double* __restrict__ sites, int64_t D, int gbits, Grid* out) {
    __shared__ unsigned long long part[4][32];
    unsigned long long k[4] = {~0ULL, ~0ULL, ~0ULL, ~0ULL};  // min x, min y, min ~x, min ~y
    for (int64_t i = threadIdx.x; i < D; i += blockDim.x) {
        const unsigned long long kx = ord_key(sites[2 * i]), ky = ord_key(sites[2 * i + 1]);
        k[0] = kx < k[0] ? kx : k[0];
        k[1] = ky < k[1] ? ky : k[1];
        k[2] = ~kx < k[2] ? ~kx : k[2];
        k[3] = ~ky < k[3] ? ~ky : k[3];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) k[q] = warp_min_u64(k[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) part[q][warp] = k[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) k[q] = warp_min_u64(lane < nw ? part[q][lane] : ~0ULL);
        if (lane == 0) {
            const double xmin = ord_value(k[0]), ymin = ord_value(k[1]);
            const double xmax = ord_value(~k[2]), ymax = ord_value(~k[3]);
            const double ex = xmax - xmin, ey = ymax - ymin;
            const double s = (ex > ey) ? ex : ey;
            Grid g;
            g.xmin = xmin;
            g.ymin = ymin;
            g.zero = !(s > 0.0);
            g.c = g.zero ? 0.0 : 1073741824.0 / s;
            g.shift = 30 - gbits;
            g.G = 1 << gbits;
            *out = g;
        }
    }
}

__global__ void quantize_kernel(const double* __restrict__ sites, int64_t D,
                                const Grid* __restrict__ grid, int2* __restrict__ qxy,
                                int* __restrict__ counts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    const Grid g = *grid;
    int qx = 0, qy = 0;
    if (!g.zero) {
        qx = (int)floor(__dmul_rn(__dsub_rn(sites[2 * i], g.xmin), g.c));
        qy = (int)floor(__dmul_rn(__dsub_rn(sites[2 * i + 1], g.ymin), g.c));
    }
    qxy[i] = make_int2(qx, qy);
    const int cell = (qy >> g.shift) * (g.G + 1) + (qx >> g.shift);
    atomicAdd(&counts[cell], 1);
}

// Exclusive scan of the cell counts (one CTA; the grid has at most 1025^2 cells).
__global__ void scan_kernel(const int* __restrict__ counts, int n, int* __restrict__ offsets,
                            int* __restrict__ cursor) {
    __shared__ int part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (n + T - 1) / T;
    const int lo = t * per, hi = min(n, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int k = 0; k < T; ++k) {
            const int v = part[k];
            part[k] = run;
            run += v;
        }
        offsets[n] = run;
    }
    __syncthreads();
    int run = part[t];
    for (int i = lo; i < hi; ++i) {
        offsets[i] = run;
        cursor[i] = run;
        run += counts[i];
    }
}

__global__ void scatter_kernel(const int2* __restrict__ qxy, int64_t D, const Grid* __restrict__ grid,
                               int* __restrict__ cursor, int4* __restrict__ cell_pts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    const Grid g = *grid;
    const int2 q = qxy[i];
    const int cell = (q.y >> g.shift) * (g.G + 1) + (q.x >> g.shift);
    const int pos = atomicAdd(&cursor[cell], 1);
    cell_pts[pos] = make_int4(q.x, q.y, (int)i, 0);
}

// ---- warp-wide top-q list -------------------------------------------------
// A key is (squared quantised distance, index), compared lexicographically.
// The list holds the 32 K smallest keys seen so far (K = 1 or 2 keys per
// lane): element e = h 32 + lane lives in register h of that lane.
// Candidates arrive in chunks of up to 32 (one per lane): a chunk is sorted
// across lanes by a bitonic network, reversed and merged into the top of the
// list by an element-wise minimum (the 32 K smallest of the union form a
// bitonic sequence), which a bitonic clean-up sorts again.

struct Key {
    unsigned long long d2;
    int j;
};

constexpr unsigned long long kInfD2 = ~0ULL;

__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
    return a.d2 < b.d2 || (a.d2 == b.d2 && a.j < b.j);
}

__device__ __forceinline__ Key inf_key() {
    Key k;
    k.d2 = kInfD2;
    k.j = INT_MAX;
    return k;
}

__device__ __forceinline__ Key shfl_key(const Key& k, int src) {
    Key o;
    o.d2 = __shfl_sync(0xffffffffu, k.d2, src);
    o.j = __shfl_sync(0xffffffffu, k.j, src);
    return o;
}

__device__ __forceinline__ Key shfl_xor_key(const Key& k, int m) {
    Key o;
    o.d2 = __shfl_xor_sync(0xffffffffu, k.d2, m);
    o.j = __shfl_xor_sync(0xffffffffu, k.j, m);
    return o;
}

// one compare-exchange stage across lanes: partner element e ^ jm (jm < 32);
// blocks of size kb ascending (kb >= 64 * K: the whole list ascending)
__device__ __forceinline__ void cx(Key& k, int e, int kb, int jm) {
    const Key o = shfl_xor_key(k, jm);
    const bool up = (e & kb) == 0;
    const bool lower = (e & jm) == 0;
    const bool keep_min = (lower == up);
    const bool mine_less = key_less(k, o);
    if (keep_min != mine_less) k = o;
}

// the compare-exchange of elements lane and lane + 32, both in this lane
__device__ __forceinline__ void cx_in(Key& lo, Key& hi, bool ascending) {
    if (key_less(hi, lo) == ascending) {
        const Key t = lo;
        lo = hi;
        hi = t;
    }
}

__device__ __forceinline__ void bitonic_sort32(Key& k, int lane) {
#pragma unroll
    for (int kb = 2; kb <= 32; kb <<= 1)
#pragma unroll
        for (int jm = kb >> 1; jm > 0; jm >>= 1) cx(k, lane, kb, jm);
}

// ascending sort of the 64 elements (L[0] at e = lane, L[1] at e = lane + 32)
__device__ __forceinline__ void bitonic_sort64(Key (&L)[2], int lane) {
    bitonic_sort32(L[0], lane);  // first half ascending,
#pragma unroll
    for (int kb = 2; kb <= 32; kb <<= 1)  // second half descending (e & 32 set flips `up`)
#pragma unroll
        for (int jm = kb >> 1; jm > 0; jm >>= 1) cx(L[1], lane | 32, kb, jm);
    cx_in(L[0], L[1], true);  // then one bitonic merge of 64
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int jm = 16; jm > 0; jm >>= 1) cx(L[h], lane + 32 * h, 64, jm);
}

// list (ascending, 32 K elements) <- the 32 K smallest of list and chunk
template <int K>
__device__ __forceinline__ void merge_chunk(Key (&L)[K], Key c, int lane) {
    bitonic_sort32(c, lane);
    const Key rev = shfl_key(c, 31 - lane);  // descending chunk against the top 32 of the list
    if (key_less(rev, L[K - 1])) L[K - 1] = rev;
    if constexpr (K == 2) cx_in(L[0], L[1], true);
#pragma unroll
    for (int h = 0; h < K; ++h)
#pragma unroll
        for (int jm = 16; jm > 0; jm >>= 1) cx(L[h], lane + 32 * h, 128, jm);
}

__device__ __forceinline__ unsigned long long qdist2(int ax, int ay, int bx, int by) {
    const long long dx = (long long)ax - bx, dy = (long long)ay - by;
    return (unsigned long long)(dx * dx + dy * dy);
}

constexpr int kSearchWarps = 4;

// One warp per site i: the min(m, lim) nearest sites j < lim, lim = i
// (group 0) or the first site of i's group of `group` sites.
template <int K>
__global__ void __launch_bounds__(32 * kSearchWarps) search_kernel(
    const int2* __restrict__ qxy, int64_t D, int m, int group, const Grid* __restrict__ grid,
    const int* __restrict__ offsets, const int4* __restrict__ cell_pts, int32_t* __restrict__ nbr) {
    __shared__ Key stage[kSearchWarps][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i64 = (int64_t)blockIdx.x * kSearchWarps + wid;
    if (i64 >= D) return;  // warp-uniform
    const int i = (int)i64;
    const int lim = group > 0 ? (i / group) * group : i;
    const int q = (lim < m) ? lim : m;
    int32_t* out = nbr + i64 * m;
    if (q == lim) {  // every earlier site is a neighbour
        for (int r = lane; r < m; r += 32) out[r] = (r < lim) ? r : -1;
        return;
    }
    Key L[K];
#pragma unroll
    for (int h = 0; h < K; ++h) L[h] = inf_key();
    const int2 me = qxy[i];
    Key* st = stage[wid];
    int n = 0;  // staged candidates (warp-uniform)
    auto worst = [&]() {  // element q - 1 (q is warp-uniform: no dynamic register index)
        Key src = L[0];
        if (K == 2 && q > 32) src = L[K - 1];
        return shfl_key(src, (q - 1) & 31);
    };
    // stage the lanes' candidates that beat the current q-th best; merge full chunks
    auto offer = [&](bool valid, Key k) {
        const Key w = worst();
        valid = valid && key_less(k, w);
        const unsigned mask = __ballot_sync(0xffffffffu, valid);
        if (valid) st[n + __popc(mask & ((1u << lane) - 1u))] = k;
        n += __popc(mask);
        __syncwarp();
        if (n >= 32) {
            merge_chunk<K>(L, st[lane], lane);
            __syncwarp();
            if (lane < n - 32) st[lane] = st[32 + lane];
            n -= 32;
            __syncwarp();
        }
    };
    auto flush = [&]() {
        if (n > 0) {
            const Key c = (lane < n) ? st[lane] : inf_key();
            merge_chunk<K>(L, c, lane);
            n = 0;
            __syncwarp();
        }
    };
    if (lim < kBruteLimit) {
        for (int base = 0; base < lim; base += 32) {
            const int j = base + lane;
            Key k = inf_key();
            if (j < lim) {
                const int2 o = qxy[j];
                k.d2 = qdist2(me.x, me.y, o.x, o.y);
                k.j = j;
            }
            offer(j < lim, k);
        }
        flush();
    } else {
        const Grid g = *grid;
        const int G = g.G, W = G + 1;
        const long long cs = 1LL << g.shift;
        const int cx0 = me.x >> g.shift, cy0 = me.y >> g.shift;
        for (int r = 0;; ++r) {
            for (int cy = cy0 - r; cy <= cy0 + r; ++cy) {
                if (cy < 0 || cy > G) continue;
                const bool edge_row = (cy == cy0 - r) || (cy == cy0 + r);
                const int step = (edge_row || r == 0) ? 1 : 2 * r;
                for (int cxx = cx0 - r; cxx <= cx0 + r; cxx += step) {
                    if (cxx < 0 || cxx > G) continue;
                    const int cell = cy * W + cxx;
                    const int b = offsets[cell], e = offsets[cell + 1];
                    for (int base = b; base < e; base += 32) {
                        const int p = base + lane;
                        Key k = inf_key();
                        bool valid = false;
                        if (p < e) {
                            const int4 o = cell_pts[p];
                            valid = o.z < lim;
                            k.d2 = qdist2(me.x, me.y, o.x, o.y);
                            k.j = o.z;
                        }
                        offer(valid, k);
                    }
                }
            }
            flush();
            const Key w = worst();
            if (w.d2 != kInfD2) {
                const long long bound = (long long)r * cs + 1;
                if (w.d2 < (unsigned long long)(bound * bound)) break;
            }
            if (cx0 - r <= 0 && cy0 - r <= 0 && cx0 + r >= G && cy0 + r >= G) break;
        }
    }
    // elements < q hold the q nearest; list them ascending by index (Sec. 2.2 block order)
    Key byj[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        byj[h].d2 = 0;
        byj[h].j = INT_MAX;
    }
#pragma unroll
    for (int h = 0; h < K; ++h)
        if (lane + 32 * h < q) byj[h].j = L[h].j;
    if constexpr (K == 1) {
        bitonic_sort32(byj[0], lane);
    } else {
        bitonic_sort64(byj, lane);
    }
#pragma unroll
    for (int h = 0; h < K; ++h) {
        const int r = lane + 32 * h;
        if (r < m) out[r] = (r < q) ? byj[h].j : -1;
    }
}

// Group k's conditioning row: the union of its members' rows (each ascending),
// merged by one thread with a p-way merge that drops repeats.
__global__ void group_union_kernel(const int32_t* __restrict__ per_site, int64_t D, int m, int p, int cmax,
                                   int32_t* __restrict__ cond, int32_t* __restrict__ count,
                                   int* __restrict__ overflow) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t G = (D + p - 1) / p;
    if (k >= G) return;
    const int64_t i0 = k * p;
    const int g = (int)((i0 + p < D) ? p : D - i0);
    int pos[64];
    for (int a = 0; a < g; ++a) pos[a] = 0;
    int32_t* row = cond + k * (int64_t)cmax;
    int n = 0, last = -1;
    bool over = false;
    for (;;) {
        int best = INT_MAX;
        for (int a = 0; a < g; ++a) {
            if (pos[a] < m) {
                const int v = per_site[(i0 + a) * m + pos[a]];
                if (v >= 0 && v < best) best = v;
            }
        }
        if (best == INT_MAX) break;
        for (int a = 0; a < g; ++a)  // consume every head equal to best
            if (pos[a] < m && per_site[(i0 + a) * m + pos[a]] == best) ++pos[a];
        if (best != last) {
            if (n < cmax)
                row[n] = best;
            else
                over = true;
            ++n;
            last = best;
        }
    }
    for (int r = n; r < cmax; ++r) row[r] = -1;
    if (count) count[k] = n < cmax ? n : cmax;
    if (over) atomicExch(overflow, 1);
}

// Random conditioning: Floyd's algorithm per group (one thread), then an
// insertion sort of the at most 63 indices.
__global__ void group_random_kernel(int64_t D, int p, int kk, uint64_t seed, int cmax,
                                    int32_t* __restrict__ cond, int32_t* __restrict__ count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t G = (D + p - 1) / p;
    if (k >= G) return;
    const int64_t n = k * p;
    const int take = (int)((kk < n) ? kk : n);
    int set[64];
    int have = 0;
    for (int r = 0; r < take; ++r) {
        const int64_t j = n - take + r;
        uint32_t c[4] = {(uint32_t)k, (uint32_t)r, 0x52C5u, (uint32_t)((uint64_t)k >> 32)};
        philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
        const int t = (int)(((uint64_t)c[0] * (uint64_t)(j + 1)) >> 32);
        bool dup = false;
        for (int a = 0; a < have; ++a) dup = dup || set[a] == t;
        set[have++] = dup ? (int)j : t;
    }
    for (int a = 1; a < have; ++a) {
        const int v = set[a];
        int b = a - 1;
        while (b >= 0 && set[b] > v) {
            set[b + 1] = set[b];
            --b;
        }
        set[b + 1] = v;
    }
    int32_t* row = cond + k * (int64_t)cmax;
    for (int r = 0; r < cmax; ++r) row[r] = (r < have) ? set[r] : -1;
    if (count) count[k] = have;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

__global__ void gather_kernel(const int32_t* __restrict__ perm, const double* __restrict__ sites,
                              const double* __restrict__ u, int64_t D, double* __restrict__ sites_out,
                              double* __restrict__ u_out, int* __restrict__ bad) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D) return;
    const int32_t j = perm[k];
    if (j < 0 || j >= D) {
        atomicExch(bad, 1);
        return;
    }
    sites_out[2 * k] = sites[2 * (int64_t)j];
    sites_out[2 * k + 1] = sites[2 * (int64_t)j + 1];
    if (u) u_out[k] = u[j];
}

}  // namespace

cudaError_t launch_gather(const int32_t* perm, const double* sites, const double* u, int64_t D,
                          double* sites_out, double* u_out, int* bad, cudaStream_t st) {
    if (D <= 0) return cudaSuccess;
    gather_kernel<<<(int)((D + 255) / 256), 256, 0, st>>>(perm, sites, u, D, sites_out, u_out, bad);
    return cudaGetLastError();
}

size_t knn_scratch_bytes(int64_t D) {
    const int k = grid_bits(D);
    const int64_t cells = (int64_t)((1 << k) + 1) * ((1 << k) + 1);
    return align256(sizeof(Grid)) + align256(sizeof(int2) * (size_t)D) +
           3 * align256(sizeof(int) * (size_t)(cells + 1)) + align256(sizeof(int4) * (size_t)D);
}

// The cell grid of a problem in the caller's scratch (knn_scratch_bytes(D)):
// bounding box, quantised coordinates, cell offsets and the sites sorted by cell.
struct Cells {
    Grid* grid;
    int2* qxy;
    int* offsets;
    int4* cell_pts;
};

cudaError_t build_cells(const double* sites, int64_t D, void* scratch, cudaStream_t st, Cells& out) {
    const int k = grid_bits(D);
    const int64_t cells = (int64_t)((1 << k) + 1) * ((1 << k) + 1);
    char* p = (char*)scratch;
    Grid* grid = (Grid*)p;
    p += align256(sizeof(Grid));
    int2* qxy = (int2*)p;
    p += align256(sizeof(int2) * (size_t)D);
    int* counts = (int*)p;
    p += align256(sizeof(int) * (size_t)(cells + 1));
    int* offsets = (int*)p;
    p += align256(sizeof(int) * (size_t)(cells + 1));
    int* cursor = (int*)p;
    p += align256(sizeof(int) * (size_t)(cells + 1));
    int4* cell_pts = (int4*)p;
    out = Cells{grid, qxy, offsets, cell_pts};
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)cells, st);
    if (e != cudaSuccess) return e;
    bbox_kernel<<<1, 1024, 0, st>>>(sites, D, k, grid);
    const int blocks = (int)((D + 255) / 256);
    quantize_kernel<<<blocks, 256, 0, st>>>(sites, D, grid, qxy, counts);
    scan_kernel<<<1, 1024, 0, st>>>(counts, (int)cells, offsets, cursor);
    scatter_kernel<<<blocks, 256, 0, st>>>(qxy, D, grid, cursor, cell_pts);
    return cudaGetLastError();
}

cudaError_t launch_knn(const double* sites, int64_t D, int m, int32_t* nbr, void* scratch,
                       cudaStream_t st, int group) {
    if (D <= 0 || m <= 0) return cudaSuccess;
    Cells c;
    cudaError_t e = build_cells(sites, D, scratch, st, c);
    if (e != cudaSuccess) return e;
    const int blocks_s = (int)((D + kSearchWarps - 1) / kSearchWarps);
    if (m <= 32)
        search_kernel<1><<<blocks_s, 32 * kSearchWarps, 0, st>>>(c.qxy, D, m, group, c.grid, c.offsets,
                                                                  c.cell_pts, nbr);
    else
        search_kernel<2><<<blocks_s, 32 * kSearchWarps, 0, st>>>(c.qxy, D, m, group, c.grid, c.offsets,
                                                                  c.cell_pts, nbr);
    return cudaGetLastError();
}

// ---- exact maxmin ordering (one persistent CTA) ----------------------------
// Same rule as the host ordering: first the site nearest the centre of the
// quantised bounding box (2q - qmax, smallest squared distance, ties to the
// smaller index), then repeatedly the unchosen site whose squared distance to
// the chosen set is largest (ties to the smaller index).  mind[i] holds that
// distance (-1 once chosen); a 32-ary tournament tree over (mind, index) gives
// the next pick at its root.  A pick at max distance r^2 can only lower the
// mind of sites closer than r, so each step scans the grid cells within r of
// the pick and recomputes the tree nodes above the leaves that changed.

constexpr int kMmThreads = 1024;
constexpr int kMmMaxLevels = 8;

struct MmTree {
    long long* val;   // node values, all levels (level l at off[l])
    int* idx;         // node argmax index
    int* flag;        // dirty marks
    int* list[2];     // dirty node lists (alternating)
    int off[kMmMaxLevels + 1];
    int n[kMmMaxLevels + 1];  // n[0] = D leaves, n[l] nodes of level l
    int levels;               // root = level `levels`, node 0
    int total;                // nodes of all levels
    int in_smem;              // 1: the arrays live in the CTA's dynamic shared memory
};

__device__ __forceinline__ bool mm_better(long long va, int ia, long long vb, int ib) {
    return va > vb || (va == vb && ia < ib);
}

__device__ __forceinline__ void mm_warp_argmax(long long& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (mm_better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
}

// Bytes of the tree arrays (8 + 4 + 4 per node, two lists of level-1 size).
__host__ __device__ inline size_t mm_tree_bytes(int total, int n1) {
    return (size_t)total * 16 + (size_t)2 * n1 * 4 + 64;
}

// Node `node` of level l (>= 1): argmax of its 32 children; lane 0 stores it,
// clears its mark and queues its parent.
__device__ __forceinline__ void mm_node(MmTree& T, const long long* mind, int l, int node, int* cnt, int lane) {
    const int c = node * 32 + lane;
    long long v = LLONG_MIN;
    int i = INT_MAX;
    if (c < T.n[l - 1]) {
        if (l == 1) {
            v = mind[c];
            i = c;
        } else {
            v = T.val[T.off[l - 1] + c];
            i = T.idx[T.off[l - 1] + c];
        }
    }
    mm_warp_argmax(v, i);
    if (lane == 0) {
        T.val[T.off[l] + node] = v;
        T.idx[T.off[l] + node] = i;
        T.flag[T.off[l] + node] = 0;
        if (l < T.levels) {
            const int parent = node >> 5;
            if (atomicExch(&T.flag[T.off[l + 1] + parent], 1) == 0)
                T.list[(l + 1) & 1][atomicAdd(&cnt[l + 1], 1)] = parent;
        }
    }
}

__global__ void __launch_bounds__(kMmThreads) maxmin_kernel(const Grid* __restrict__ grid,
                                                            const int2* __restrict__ qxy,
                                                            const int* __restrict__ offsets,
                                                            const int4* __restrict__ cell_pts, int D,
                                                            long long* __restrict__ mind, MmTree T,
                                                            int32_t* __restrict__ perm) {
    extern __shared__ __align__(16) unsigned char mm_smem[];
    __shared__ long long red_v[kMmThreads / 32], red_y[kMmThreads / 32];
    __shared__ int red_i[kMmThreads / 32];
    __shared__ int cnt[kMmMaxLevels + 2];
    __shared__ int s_pick;
    __shared__ long long s_r2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Grid g = *grid;
    const int W = g.G + 1;
    if (T.in_smem) {  // carve the tree out of dynamic shared memory
        unsigned char* p = mm_smem;
        T.val = (long long*)p;
        p += (size_t)T.total * 8;
        T.idx = (int*)p;
        p += (size_t)T.total * 4;
        T.flag = (int*)p;
        p += (size_t)T.total * 4;
        T.list[0] = (int*)p;
        p += (size_t)T.n[1] * 4;
        T.list[1] = (int*)p;
    }

    // leaves at "infinity", no marks
    for (int i = tid; i < D; i += kMmThreads) mind[i] = LLONG_MAX;
    for (int x = tid; x < T.total; x += kMmThreads) T.flag[x] = 0;
    // the first site: nearest the centre of the quantised bounding box
    long long qxm = 0, qym = 0;
    for (int i = tid; i < D; i += kMmThreads) {
        qxm = max(qxm, (long long)qxy[i].x);
        qym = max(qym, (long long)qxy[i].y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        qxm = max(qxm, __shfl_xor_sync(0xffffffffu, qxm, o));
        qym = max(qym, __shfl_xor_sync(0xffffffffu, qym, o));
    }
    if (lane == 0) {
        red_v[warp] = qxm;
        red_y[warp] = qym;
    }
    __syncthreads();
    qxm = 0;
    qym = 0;
    for (int w = 0; w < kMmThreads / 32; ++w) {
        qxm = max(qxm, red_v[w]);
        qym = max(qym, red_y[w]);
    }
    __syncthreads();
    long long bv = LLONG_MAX;
    int bi = INT_MAX;
    for (int i = tid; i < D; i += kMmThreads) {
        const long long dx = 2LL * qxy[i].x - qxm, dy = 2LL * qxy[i].y - qym;
        const long long v = dx * dx + dy * dy;
        if (v < bv || (v == bv && i < bi)) {
            bv = v;
            bi = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {  // arg-min over (distance, index)
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov < bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        red_v[warp] = bv;
        red_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
        long long v = LLONG_MAX;
        int f = INT_MAX;
        for (int w = 0; w < kMmThreads / 32; ++w)
            if (red_v[w] < v || (red_v[w] == v && red_i[w] < f)) {
                v = red_v[w];
                f = red_i[w];
            }
        perm[0] = f;
        mind[f] = -1;
        s_pick = f;
        s_r2 = LLONG_MAX;  // every site is within reach of the first pick
        for (int l = 0; l < kMmMaxLevels + 2; ++l) cnt[l] = 0;
        T.flag[T.off[1] + (f >> 5)] = 1;
        T.list[1][0] = f >> 5;
        cnt[1] = 1;
    }
    __syncthreads();

    for (int k = 1; k < D; ++k) {
        // scan: lower mind of the sites within reach of the last pick
        const int pick = s_pick;
        const long long r2 = s_r2;
        const int2 pq = qxy[pick];
        int cx_lo = 0, cx_hi = g.G, cy_lo = 0, cy_hi = g.G;
        if (r2 != LLONG_MAX) {
            const long long rr = (long long)sqrt((double)r2) + 1;  // |dx|, |dy| < rr for d^2 < r2
            cx_lo = (int)(max(0LL, (long long)pq.x - rr) >> g.shift);
            cy_lo = (int)(max(0LL, (long long)pq.y - rr) >> g.shift);
            cx_hi = (int)min((long long)g.G, ((long long)pq.x + rr) >> g.shift);
            cy_hi = (int)min((long long)g.G, ((long long)pq.y + rr) >> g.shift);
        }
        for (int row = cy_lo + warp; row <= cy_hi; row += kMmThreads / 32) {
            const int b = offsets[row * W + cx_lo], e = offsets[row * W + cx_hi + 1];
            for (int x = b + lane; x < e; x += 32) {
                const int4 o = cell_pts[x];
                const long long mi = mind[o.z];
                if (mi < 0) continue;
                const long long dx = (long long)o.x - pq.x, dy = (long long)o.y - pq.y;
                const long long d2 = dx * dx + dy * dy;
                if (d2 < mi) {
                    mind[o.z] = d2;
                    const int node = o.z >> 5;
                    if (atomicExch(&T.flag[T.off[1] + node], 1) == 0) T.list[1][atomicAdd(&cnt[1], 1)] = node;
                }
            }
        }
        __syncthreads();
        // level 1 by all warps
        for (int j = warp; j < cnt[1]; j += kMmThreads / 32) mm_node(T, mind, 1, T.list[1][j], cnt, lane);
        __syncthreads();
        // upper levels and the next pick by warp 0
        if (warp == 0) {
            for (int l = 2; l <= T.levels; ++l) {
                const int n = cnt[l];
                for (int j = 0; j < n; ++j) mm_node(T, mind, l, T.list[l & 1][j], cnt, lane);
                __syncwarp();
            }
            if (lane == 0) {
                const int root = T.off[T.levels];
                const int nxt = T.idx[root];
                perm[k] = nxt;
                mind[nxt] = -1;
                s_pick = nxt;
                s_r2 = T.val[root];
                for (int l = 0; l < kMmMaxLevels + 2; ++l) cnt[l] = 0;
                T.flag[T.off[1] + (nxt >> 5)] = 1;  // its own leaf changed
                T.list[1][0] = nxt >> 5;
                cnt[1] = 1;
            }
        }
        __syncthreads();
    }
}

// Tree shape for D leaves: level sizes and offsets.
bool mm_shape(int64_t D, MmTree& T) {
    T.n[0] = (int)D;
    T.off[0] = 0;
    int levels = 0, total = 0;
    int64_t n = D;
    do {
        n = (n + 31) / 32;
        ++levels;
        if (levels > kMmMaxLevels) return false;
        T.off[levels] = total;
        T.n[levels] = (int)n;
        total += (int)n;
    } while (n > 1);
    T.levels = levels;
    T.total = total;
    return true;
}

constexpr size_t kMmSmemMax = 200 * 1024;

size_t maxmin_scratch_bytes(int64_t D) {
    MmTree T;
    if (!mm_shape(D, T)) return 0;
    return knn_scratch_bytes(D) + align256(sizeof(long long) * (size_t)D) + align256(mm_tree_bytes(T.total, T.n[1]));
}

cudaError_t launch_maxmin(const double* sites, int64_t D, int32_t* perm, void* scratch, cudaStream_t st) {
    if (D <= 0) return cudaSuccess;
    MmTree T;
    if (!mm_shape(D, T)) return cudaErrorInvalidValue;
    Cells c;
    cudaError_t e = build_cells(sites, D, scratch, st, c);
    if (e != cudaSuccess) return e;
    char* p = (char*)scratch + knn_scratch_bytes(D);
    long long* mind = (long long*)p;
    p += align256(sizeof(long long) * (size_t)D);
    const size_t tree = mm_tree_bytes(T.total, T.n[1]);
    T.in_smem = tree <= kMmSmemMax;
    size_t smem = 0;
    if (T.in_smem) {
        smem = tree;
        static std::mutex mu;
        static std::map<int, size_t> attr;
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        if (smem > 48 * 1024 && attr[dev] < smem) {
            e = cudaFuncSetAttribute(maxmin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmSmemMax);
            if (e != cudaSuccess) return e;
            attr[dev] = kMmSmemMax;
        }
        T.val = nullptr;
        T.idx = T.flag = T.list[0] = T.list[1] = nullptr;
    } else {
        T.val = (long long*)p;
        p += (size_t)T.total * 8;
        T.idx = (int*)p;
        p += (size_t)T.total * 4;
        T.flag = (int*)p;
        p += (size_t)T.total * 4;
        T.list[0] = (int*)p;
        p += (size_t)T.n[1] * 4;
        T.list[1] = (int*)p;
    }
    maxmin_kernel<<<1, kMmThreads, smem, st>>>(c.grid, c.qxy, c.offsets, c.cell_pts, (int)D, mind, T, perm);
    return cudaGetLastError();
}

// ---- XY ordering on the device (D <= 8192) ----------------------------------
// The rank of site i in the (x, y, index) order is the number of sites whose
// key is smaller (the host's XY rule; keys are unique through the index);
// perm[rank_i] = i.

constexpr int kXyMax = 8192;
constexpr int kXyThreads = 256;

// Grid (site blocks x chunks of the other sites): each thread counts, for its
// site, the smaller keys of one chunk and adds the count to rank[i] (integer
// adds: the total does not depend on their order).
constexpr int kXyChunk = 128;  // 20 chunks at D = 2,500: a CTA for every SM

__global__ void __launch_bounds__(kXyThreads) order_xy_rank_kernel(const double* __restrict__ sites, int D,
                                                                   int* __restrict__ rank) {
    __shared__ unsigned long long tx[kXyChunk], ty[kXyChunk];
    const int i = blockIdx.x * kXyThreads + threadIdx.x;
    const int j0 = blockIdx.y * kXyChunk;
    const int n = min(kXyChunk, D - j0);
    for (int t = threadIdx.x; t < n; t += kXyThreads) {
        tx[t] = ord_key(sites[2 * (j0 + t)]);
        ty[t] = ord_key(sites[2 * (j0 + t) + 1]);
    }
    __syncthreads();
    if (i >= D) return;
    const unsigned long long xi = ord_key(sites[2 * i]), yi = ord_key(sites[2 * i + 1]);
    int cnt = 0;
    for (int t = 0; t < n; ++t) {
        const unsigned long long xj = tx[t], yj = ty[t];
        cnt += (xj < xi) || (xj == xi && (yj < yi || (yj == yi && j0 + t < i)));
    }
    if (cnt) atomicAdd(&rank[i], cnt);
}

__global__ void order_xy_scatter_kernel(const int* __restrict__ rank, int D, int32_t* __restrict__ perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < D) perm[rank[i]] = i;
}

size_t order_xy_scratch_bytes(int64_t D) { return sizeof(int) * (size_t)(D > 0 ? D : 1); }

cudaError_t launch_order_xy(const double* sites, int64_t D, int32_t* perm, void* scratch, cudaStream_t st) {
    if (D <= 0 || D > kXyMax) return cudaErrorInvalidValue;
    int* rank = (int*)scratch;
    cudaError_t e = cudaMemsetAsync(rank, 0, sizeof(int) * (size_t)D, st);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((D + kXyThreads - 1) / kXyThreads), (unsigned)((D + kXyChunk - 1) / kXyChunk));
    order_xy_rank_kernel<<<grid, kXyThreads, 0, st>>>(sites, (int)D, rank);
    order_xy_scatter_kernel<<<(unsigned)((D + 255) / 256), 256, 0, st>>>(rank, (int)D, perm);
    return cudaGetLastError();
}

cudaError_t launch_group_union(const int32_t* per_site, int64_t D, int m, int p, int cmax, int32_t* cond,
                               int32_t* count, int* overflow, cudaStream_t st) {
    const int64_t G = (D + p - 1) / p;
    if (G <= 0) return cudaSuccess;
    group_union_kernel<<<(int)((G + 127) / 128), 128, 0, st>>>(per_site, D, m, p, cmax, cond, count, overflow);
    return cudaGetLastError();
}

// The largest number of leading non-negative entries over G rows of width m.
__global__ void rows_max_kernel(const int32_t* __restrict__ rows, int64_t G, int m, int* __restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G) return;
    const int32_t* row = rows + k * (int64_t)m;
    int c = 0;
    while (c < m && row[c] >= 0) ++c;
    atomicMax(out, c);
}

cudaError_t launch_rows_max(const int32_t* rows, int64_t G, int m, int* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), st);
    if (e != cudaSuccess || G <= 0 || m <= 0) return e;
    rows_max_kernel<<<(int)((G + 255) / 256), 256, 0, st>>>(rows, G, m, out);
    return cudaGetLastError();
}

cudaError_t launch_group_random(int64_t D, int p, int kk, uint64_t seed, int cmax, int32_t* cond,
                                int32_t* count, cudaStream_t st) {
    const int64_t G = (D + p - 1) / p;
    if (G <= 0) return cudaSuccess;
    group_random_kernel<<<(int)((G + 127) / 128), 128, 0, st>>>(D, p, kk, seed, cmax, cond, count);
    return cudaGetLastError();
}

}  // namespace vk
