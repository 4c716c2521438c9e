// vk_internal.h -- declarations shared by the translation units of libvecchia
// (host API, neighbour kernels, Genz kernels).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <vector>

#include "vecchia.h"

namespace vk {

// Bucketed block sizes: a site with q neighbours has d = q + 1 <= 32
// variables; its problem's Genz kernel is instantiated for the smallest
// DMAX >= m + 1.  The buckets put m = 8, 12, 16, 20, 24, 28 at the top of
// theirs, so a lane keeps exactly m partial sums in registers there.
constexpr int kNumBuckets = 7;
constexpr int kDmaxBuckets[kNumBuckets] = {9, 13, 17, 21, 25, 29, 32};
constexpr int kMaxS = VECCHIA_MAX_S;
constexpr int kMaxDim = 32;  // lattice coordinates per problem (q <= 31)

inline int bucket_of(int d) {
    for (int b = 0; b < kNumBuckets; ++b)
        if (d <= kDmaxBuckets[b]) return b;
    return -1;
}

struct ProbResult;

// One log-CDF problem as the device sees it (all pointers device memory).
struct ProbDev {
    const double* sites;   // D x 2, ordered
    const int32_t* nbr;    // D x m
    const double* u;       // D
    double* num;           // D x S partial means (output)
    double* den;           // D x S
    const uint32_t* g;     // lattice vector, >= m entries
    const double* delta;   // S x dim shifts (FP64)
    const uint32_t* gfix;  // round(g_j 2^32 / N)            (mixed path)
    const uint32_t* dfix;  // top 32 bits of the shift         (mixed path), S x dim
    int64_t D;
    int64_t N;
    double variance, range, nu, nugget;
    int32_t cov_kind;
    int32_t m;
    int32_t S;
    int32_t dim;           // row stride of delta / dfix
    ProbResult* res;       // result slot owned by the caller (segment calls), or nullptr
};

// Result slot of a problem, written by the log-sum kernel.
struct ProbResult {
    double log_p;
    double std_err;
    int64_t bad_site;      // first failing ordered site (INT64_MAX if none)
    int32_t status;        // VECCHIA_OK or an error code
    int32_t pad;
};

// Launch tile of the Genz kernel.
struct GenzTile {
    int warps;      // warps per CTA (1..16)
    int points;     // points per lane per pass (1, 2 or 4): template parameter
    int slices;     // lattice slices per shift, spread over the CTA's warps
    int groups;     // shift groups per site, spread over CTAs (N x S split)
};

// ---------------- kernels' host launchers (genz.cu, knn.cu) ----------------

// Genz partial sums for the sites of one DMAX bucket, given as segments:
// segment k = sites seg_base[k].y .. of problem seg_base[k].x, with
// seg_prefix (n_segs + 1 entries, device) the running site count.
cudaError_t launch_genz(int bucket, bool mixed, const GenzTile& tile, const ProbDev* probs,
                        const int* seg_prefix, const int2* seg_base, int n_segs, int n_sites,
                        ProbResult* results, int* fallback_count, int2* fallback_items, int max_S,
                        cudaStream_t st);
// FP64 re-evaluation of the items the mixed kernel flagged (device-side count).
cudaError_t launch_genz_fallback(const ProbDev* probs, const int* fallback_count,
                                 const int2* fallback_items, int capacity, ProbResult* results,
                                 cudaStream_t st);
// Per-problem deterministic log-sum and standard error; writes results and
// terms.  scratch_off[p] points at logsum_scratch(D_p, S_p) doubles.
inline int64_t logsum_slices(int64_t D) { return (D + 255) / 256; }
inline int64_t logsum_scratch(int64_t D, int S) { return logsum_slices(D) * (S + 1); }
cudaError_t launch_logsum(const ProbDev* probs, int n_probs, int max_slices, ProbResult* results,
                          double* const* terms, double* scratch, const int64_t* scratch_off,
                          cudaStream_t st);
// Shift tables on the device: delta (S x dim FP64) and dfix (S x dim uint32).
cudaError_t launch_shifts(const uint64_t* seeds, const int32_t* S, const int64_t* out_off,
                          int n_probs, int dim, double* delta, uint32_t* dfix, cudaStream_t st);
cudaError_t launch_init_results(ProbResult* results, int n, int* fallback_count, cudaStream_t st);

// Neighbour search for one problem (sites ordered, device); scratch from the
// caller's arena (bytes from knn_scratch_bytes).
size_t knn_scratch_bytes(int64_t D);
cudaError_t launch_knn(const double* sites, int64_t D, int m, int32_t* nbr, void* scratch,
                       cudaStream_t st);

// sites_out[k] = sites[perm[k]], u_out[k] = u[perm[k]]; *bad = 1 on an index out of range.
cudaError_t launch_gather(const int32_t* perm, const double* sites, const double* u, int64_t D,
                          double* sites_out, double* u_out, int* bad, cudaStream_t st);

// The FP32 special functions of the mixed path on n device values (diagnostic).
cudaError_t launch_eval_special(int which, const float* x, int64_t n, float* out, cudaStream_t st);

int device_sm_count(int device);

}  // namespace vk
