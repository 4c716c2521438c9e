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

// Bucketed block sizes: a term with d variables (d = q + 1 for a site with q
// neighbours; d = c + p for a group of p sites conditioned on c) is evaluated
// by the Genz kernel instantiated for the smallest DMAX >= its problem's
// largest d.  Up to 32 the buckets put m = 8, 12, ..., 28 at the top of
// theirs (a lane keeps exactly m partial sums in registers there); 48 and 64
// take the paper's m = 30 ... 50 and joint groups.
constexpr int kNumBuckets = 9;
constexpr int kDmaxBuckets[kNumBuckets] = {9, 13, 17, 21, 25, 29, 32, 48, 64};
constexpr int kMaxS = VECCHIA_MAX_S;
constexpr int kMaxDim = 64;  // lattice coordinates per term (d - 1 <= 63)

inline int bucket_of(int d) {
    for (int b = 0; b < kNumBuckets; ++b)
        if (d <= kDmaxBuckets[b]) return b;
    return -1;
}

// Largest term dimension of a problem: m + 1 (classic), m + p (groups of p).
inline int max_term_dim(int m, int group) { return group > 0 ? m + group : m + 1; }
// The same for a problem whose group rows hold at most cond_max sites (0: m).
inline int max_term_dim(int m, int group, int cond_max) {
    return max_term_dim((group > 0 && cond_max > 0 && cond_max < m) ? cond_max : m, group);
}
// Number of Vecchia terms: one per site (classic) or per group of p sites.
inline int64_t n_terms_of(int64_t D, int group) { return group > 0 ? (D + group - 1) / group : D; }

struct ProbResult;

// One log-CDF problem as the device sees it (all pointers device memory).
struct ProbDev {
    const double* sites;   // D x 2, ordered
    const int32_t* nbr;    // n_terms x m conditioning rows (classic: N_i)
    const double* u;       // D
    double* num;           // n_terms x S partial means (output)
    double* den;           // n_terms x S
    const uint32_t* g;     // lattice vector, >= m entries
    const double* delta;   // S x dim shifts (FP64)
    const uint32_t* gfix;  // round(g_j 2^32 / N)            (mixed path)
    const uint32_t* dfix;  // top 32 bits of the shift         (mixed path), S x dim
    int64_t D;
    int64_t n_terms;       // D (classic) or ceil(D / group)
    int64_t N;
    double variance, range, nu, nugget;
    double cos_a, sin_a, aspect;  // anisotropic exponential: rotation and aspect ratio
    const double* lr_V;    // low-rank correction of the covariance (or nullptr): D x lr_k,
    double lr_scale;       //   entry (a, b) -= lr_scale * V_a . V_b  (conditional covariance)
    int32_t cov_kind;
    int32_t m;
    int32_t group;         // 0: classic (term i = site i, N_i = min(m, i) nearest); p: groups of p
    int32_t lr_k;          // columns of lr_V (0: no correction)
    int32_t S;
    int32_t dim;           // row stride of delta / dfix
    ProbResult* res;       // result slot owned by the caller (segment calls), or nullptr
};

// Result slot of a problem, written by the log-sum kernel.
struct ProbResult {
    double log_p;
    double std_err;
    int64_t bad_site;      // first failing term (ordered site, or group) (INT64_MAX if none)
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

// Genz partial sums for the terms of one DMAX bucket, given as segments:
// segment k = terms seg_base[k].y .. of problem seg_base[k].x, with
// seg_prefix (n_segs + 1 entries, device) the running term count.
cudaError_t launch_genz(int bucket, bool mixed, const GenzTile& tile, const ProbDev* probs,
                        const int* seg_prefix, const int2* seg_base, int n_segs, int n_sites,
                        ProbResult* results, int* fallback_count, int2* fallback_items, int max_S,
                        int fb_capacity, cudaStream_t st);
// Entries to add to a flagged-item list beyond (sites x shift groups): a launch
// may cut its last round into smaller items, at most one grid's worth (of at
// most 32 CTAs per SM) per bucket.
inline int64_t genz_items_slack(int sm_count) { return (int64_t)kNumBuckets * 32 * sm_count; }
// Log-space re-evaluation of the items the mixed kernel flagged (device-side
// count), instantiated for the largest bucket of the batch.
cudaError_t launch_genz_fallback(int max_bucket, const ProbDev* probs, const int* fallback_count,
                                 const int2* fallback_items, int capacity, ProbResult* results,
                                 int max_S, cudaStream_t st);
// Per-problem deterministic log-sum and standard error over its n_terms terms;
// writes results and terms.  scratch_off[p] points at logsum_scratch(n_terms_p, S_p) doubles.
constexpr int kLogsumSlice = 32;  // sites per CTA of the log-sum's first pass
inline int64_t logsum_slices(int64_t D) { return (D + kLogsumSlice - 1) / kLogsumSlice; }
inline int64_t logsum_scratch(int64_t D, int S) { return logsum_slices(D) * (S + 1); }
cudaError_t launch_logsum(const ProbDev* probs, int n_probs, int max_slices, ProbResult* results,
                          double* const* terms, double* scratch, const int64_t* scratch_off,
                          cudaStream_t st);
// Shift tables on the device: delta (S x dim FP64) and dfix (S x dim uint32).
cudaError_t launch_shifts(const uint64_t* seeds, const int32_t* S, const int64_t* out_off,
                          int n_probs, int dim, double* delta, uint32_t* dfix, cudaStream_t st);
cudaError_t launch_init_results(ProbResult* results, int n, int* fallback_count, cudaStream_t st);

// Neighbour search for one problem (sites ordered, device); scratch from the
// caller's arena (bytes from knn_scratch_bytes).  group = 0: the min(m, i)
// nearest j < i of every site i; group = p: the min(m, i0) nearest j < i0,
// i0 = (i / p) p the first site of i's group.  m <= 63.
size_t knn_scratch_bytes(int64_t D);
cudaError_t launch_knn(const double* sites, int64_t D, int m, int32_t* nbr, void* scratch,
                       cudaStream_t st, int group = 0);
// Exact maxmin ordering on the device (one persistent CTA); perm (D, device)
// gets new position -> old index; scratch from maxmin_scratch_bytes(D).
size_t maxmin_scratch_bytes(int64_t D);
cudaError_t launch_maxmin(const double* sites, int64_t D, int32_t* perm, void* scratch, cudaStream_t st);
// XY ordering (x, then y, then index) of D <= 8192 device sites (ranks by counting).
size_t order_xy_scratch_bytes(int64_t D);
cudaError_t launch_order_xy(const double* sites, int64_t D, int32_t* perm, void* scratch, cudaStream_t st);
constexpr int64_t kOrderXyDeviceMax = 8192;
// Union of the members' sets (per_site: D x m from launch_knn with group p)
// into ascending rows of cond (n_groups x cmax, -1 padded) and count; *overflow
// = 1 if a union has more than cmax entries.
cudaError_t launch_group_union(const int32_t* per_site, int64_t D, int m, int p, int cmax, int32_t* cond,
                               int32_t* count, int* overflow, cudaStream_t st);
// Random conditioning rows: a uniform subset of min(kk, k p) sites before
// group k (Floyd's algorithm on Philox4x32-10 draws), ascending.
// *out = the largest number of leading non-negative entries over G rows of width m.
cudaError_t launch_rows_max(const int32_t* rows, int64_t G, int m, int* out, cudaStream_t st);
cudaError_t launch_group_random(int64_t D, int p, int kk, uint64_t seed, int cmax, int32_t* cond,
                                int32_t* count, cudaStream_t st);

// Covariance of D device sites (FP64, lower triangle of the D x D array A) and
// its blocked Cholesky factor in place; *bad = min failing row (start INT_MAX).
// With tc_scratch (chol_tc_scratch_bytes(D) bytes) the trailing updates run on
// the tensor cores at FP64 accuracy (chol_tc.cu); a device wait of theirs that
// runs out sets *timeout.
cudaError_t launch_cov_chol(const double* sites, int64_t D, const vecchia_cov& cov, double* A, int* bad,
                            cudaStream_t st, void* tc_scratch = nullptr, int* timeout = nullptr,
                            uint64_t wait_ns = 2000000000ull);
// The tensor-core trailing update (chol_tc.cu): a panel's rows as 7 bf16
// digit matrices per group of 8 rows (kCholSliceGroupBytes a group) and their
// exponents, written by the row solve; part 0 updates the next block column,
// part 1 the rest of the trailing matrix below base.
constexpr int kCholSlices = 7;
constexpr uint32_t kCholSliceGroupBytes = kCholSlices * 512;
size_t chol_tc_slice_bytes(int64_t D);
size_t chol_tc_scratch_bytes(int64_t D);
// Once per device, outside any stream capture: the update kernel's attributes.
cudaError_t chol_tc_prepare();
cudaError_t launch_chol_update_tc(const unsigned char* sl, const int* ex, double* A, int64_t D, int64_t base,
                                  int part, int* timeout, uint64_t wait_ns, cudaStream_t st);
// Conditioning on observed sites (censor.cu): with L the Cholesky factor of
// Sigma_II (k x k, from launch_cov_chol on sites_i), rows a < nc of V
// ((nc + 1) x k) get L^-1 Sigma_{I a}, row nc gets w = L^-1 x_I, and
// u_out[a] = x_c[a] - V_a . w (the censored thresholds minus the conditional mean).
cudaError_t launch_conditioning(const double* L, int k, const double* sites_i, const double* x_i,
                                const double* sites_c, const double* x_c, int64_t nc, const vecchia_cov& cov,
                                double* V, double* u_out, cudaStream_t st);

// Full D-dimensional Genz estimate (full.cu): covariance, blocked FP64
// Cholesky, Genz over all variables; part_host gets S x ceil(N/128) tile sums
// of the point products, *bad_host the first non-positive pivot (INT_MAX if none).
size_t full_genz_scratch_bytes(int64_t D, int64_t N, int S, bool mixed);
// Point-block sums per shift written by launch_full_genz.
int64_t full_genz_blocks_per_shift(int64_t N, bool mixed);
// part_host: per-shift point-block sums (S x full_genz_blocks_per_shift); bad_host:
// the first failing pivot (INT_MAX if none); timeout_host: nonzero if a device
// wait of the tensor-core kernel ran out; ev_begin / ev_end (may be null) are
// recorded around the recursion kernel alone.
cudaError_t launch_full_genz(const double* sites, const double* u, int64_t D, const vecchia_cov& cov, int64_t N,
                             int S, bool mixed, const uint32_t* g_host, const uint32_t* gfix_host,
                             uint64_t seed, void* scratch, double* part_host, int* bad_host, int* timeout_host,
                             uint64_t wait_ns, int withhold, cudaEvent_t ev_begin, cudaEvent_t ev_end,
                             cudaStream_t st);
// The mixed recursion on the tensor cores (full_tc.cu), given the FP64 factor A.
// wait_ns: limit of its progress waits (0: the built-in 2 s); withhold: the
// copy lane issues nothing (tests of the timeout path only).
size_t full_tc_scratch_bytes(int64_t D, int64_t N, int S);
int64_t full_tc_blocks_per_shift(int64_t N);
cudaError_t launch_full_genz_tc(const double* A, const double* u, int64_t D, int64_t N, int S, const uint32_t* gfix,
                                const uint32_t* dfix, int dim, void* scratch, double* part, int* timeout,
                                uint64_t wait_ns, int withhold, cudaEvent_t ev_begin, cudaEvent_t ev_end,
                                cudaStream_t st);

// sites_out[k] = sites[perm[k]], u_out[k] = u[perm[k]]; *bad = 1 on an index out of range.
cudaError_t launch_gather(const int32_t* perm, const double* sites, const double* u, int64_t D,
                          double* sites_out, double* u_out, int* bad, cudaStream_t st);

// The FP32 special functions of the mixed path on n device values (diagnostic).
cudaError_t launch_eval_special(int which, const float* x, int64_t n, float* out, cudaStream_t st);
cudaError_t launch_eval_special64(int which, const double* x, int64_t n, double* out, cudaStream_t st);

int device_sm_count(int device);

#ifdef __CUDACC__
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 bijection with
// the Weyl key schedule, in place on the counter.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}
#endif

}  // namespace vk
