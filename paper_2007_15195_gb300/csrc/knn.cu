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
//   - per site, visit rings of cells of growing Chebyshev radius r around the
//     site's cell, keeping the best q keys among sites j < i; after ring r every
//     unvisited site is at least r*cell + 1 away in one coordinate, so the
//     search stops once the q-th best squared distance is below (r*cell + 1)^2;
//   - sites with a small index are searched by brute force over j < i.
#include <climits>

#include "vk_internal.h"

namespace vk {
namespace {

constexpr int kMaxQ = 32;
constexpr int kBruteLimit = 2048;

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

__global__ void bbox_kernel(const double* __restrict__ sites, int64_t D, int gbits, Grid* out) {
    __shared__ double sx0[1024], sx1[1024], sy0[1024], sy1[1024];
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int64_t i = threadIdx.x; i < D; i += blockDim.x) {
        const double x = sites[2 * i], y = sites[2 * i + 1];
        x0 = fmin(x0, x);
        x1 = fmax(x1, x);
        y0 = fmin(y0, y);
        y1 = fmax(y1, y);
    }
    const int t = threadIdx.x;
    sx0[t] = x0;
    sx1[t] = x1;
    sy0[t] = y0;
    sy1[t] = y1;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            sx0[t] = fmin(sx0[t], sx0[t + o]);
            sx1[t] = fmax(sx1[t], sx1[t + o]);
            sy0[t] = fmin(sy0[t], sy0[t + o]);
            sy1[t] = fmax(sy1[t], sy1[t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const double ex = sx1[0] - sx0[0], ey = sy1[0] - sy0[0];
        const double s = (ex > ey) ? ex : ey;
        Grid g;
        g.xmin = sx0[0];
        g.ymin = sy0[0];
        g.zero = !(s > 0.0);
        g.c = g.zero ? 0.0 : 1073741824.0 / s;
        g.shift = 30 - gbits;
        g.G = 1 << gbits;
        *out = g;
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

struct TopQ {
    long long kd[kMaxQ];
    int kj[kMaxQ];
    int n, q;

    __device__ __forceinline__ void consider(long long d2, int j) {
        if (n == q) {
            const long long wd = kd[q - 1];
            if (d2 > wd || (d2 == wd && j > kj[q - 1])) return;
        }
        int pos = (n < q) ? n : q - 1;
        if (n < q) ++n;
        while (pos > 0 && (kd[pos - 1] > d2 || (kd[pos - 1] == d2 && kj[pos - 1] > j))) {
            kd[pos] = kd[pos - 1];
            kj[pos] = kj[pos - 1];
            --pos;
        }
        kd[pos] = d2;
        kj[pos] = j;
    }
};

__device__ __forceinline__ long long qdist2(int ax, int ay, int bx, int by) {
    const long long dx = (long long)ax - bx, dy = (long long)ay - by;
    return dx * dx + dy * dy;
}

__global__ void __launch_bounds__(128) search_kernel(const int2* __restrict__ qxy, int64_t D, int m,
                                                     const Grid* __restrict__ grid,
                                                     const int* __restrict__ offsets,
                                                     const int4* __restrict__ cell_pts,
                                                     int32_t* __restrict__ nbr) {
    const int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i64 >= D) return;
    const int i = (int)i64;
    const int q = (i < m) ? i : m;
    int32_t* out = nbr + i64 * m;
    if (q == i) {  // every previous site is a neighbour
        for (int r = 0; r < m; ++r) out[r] = (r < i) ? r : -1;
        return;
    }
    TopQ top;
    top.n = 0;
    top.q = q;
    const int2 me = qxy[i];
    if (i < kBruteLimit) {
        for (int j = 0; j < i; ++j) {
            const int2 o = qxy[j];
            top.consider(qdist2(me.x, me.y, o.x, o.y), j);
        }
    } else {
        const Grid g = *grid;
        const int G = g.G, W = G + 1;
        const long long cs = 1LL << g.shift;
        const int cx0 = me.x >> g.shift, cy0 = me.y >> g.shift;
        for (int r = 0;; ++r) {
            for (int cy = cy0 - r; cy <= cy0 + r; ++cy) {
                if (cy < 0 || cy > G) continue;
                const bool edge_row = (cy == cy0 - r) || (cy == cy0 + r);
                const int step = edge_row ? 1 : 2 * r;
                for (int cx = cx0 - r; cx <= cx0 + r; cx += (step > 0 ? step : 1)) {
                    if (cx < 0 || cx > G) continue;
                    const int cell = cy * W + cx;
                    const int b = offsets[cell], e = offsets[cell + 1];
                    for (int p = b; p < e; ++p) {
                        const int4 o = cell_pts[p];
                        if (o.z < i) top.consider(qdist2(me.x, me.y, o.x, o.y), o.z);
                    }
                }
            }
            if (top.n == q) {
                const long long bound = (long long)r * cs + 1;
                if (top.kd[q - 1] < bound * bound) break;
            }
            if (cx0 - r <= 0 && cy0 - r <= 0 && cx0 + r >= G && cy0 + r >= G) break;
        }
    }
    // list ascending by index (the block order of Sec. 2.2)
    for (int a = 1; a < top.n; ++a) {
        const int v = top.kj[a];
        int b = a - 1;
        while (b >= 0 && top.kj[b] > v) {
            top.kj[b + 1] = top.kj[b];
            --b;
        }
        top.kj[b + 1] = v;
    }
    for (int r = 0; r < m; ++r) out[r] = (r < top.n) ? top.kj[r] : -1;
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

cudaError_t launch_knn(const double* sites, int64_t D, int m, int32_t* nbr, void* scratch,
                       cudaStream_t st) {
    if (D <= 0 || m <= 0) return cudaSuccess;
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

    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)cells, st);
    if (e != cudaSuccess) return e;
    bbox_kernel<<<1, 1024, 0, st>>>(sites, D, k, grid);
    const int blocks = (int)((D + 255) / 256);
    quantize_kernel<<<blocks, 256, 0, st>>>(sites, D, grid, qxy, counts);
    scan_kernel<<<1, 1024, 0, st>>>(counts, (int)cells, offsets, cursor);
    scatter_kernel<<<blocks, 256, 0, st>>>(qxy, D, grid, cursor, cell_pts);
    search_kernel<<<(int)((D + 127) / 128), 128, 0, st>>>(qxy, D, m, grid, offsets, cell_pts, nbr);
    return cudaGetLastError();
}

}  // namespace vk
