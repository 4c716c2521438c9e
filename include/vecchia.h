/*
 * vecchia.h -- C ABI of libvecchia, a GB300 (sm_103a) implementation of the
 * hot path of the Vecchia approximation to a high-dimensional Gaussian CDF
 * (Nascimento & Shaby, "A Vecchia approximation for high-dimensional
 * Gaussian cumulative distribution functions arising from spatial data",
 * arXiv 2007.15195).
 *
 * The problem (Sec. 2, Eq. int): P(X < x) for X ~ N(mu, Sigma), Sigma from a
 * stationary spatial covariance at D sites.  The approximation (Sec. 2.2,
 * Eq. vecchia-cdf):
 *     log P(X < x) ~ sum_i [ log Phi_{q_i+1}(u_i, u_{N(i)}) - log Phi_{q_i}(u_{N(i)}) ],
 * q_i = min(m, i-1), N(i) the q_i nearest previously ordered sites (Sec. 2.1),
 * each low-dimensional CDF by Genz's separation-of-variables quasi-Monte Carlo
 * (Sec. 2.2, Sec. 3), each term on the log scale and then summed (Sec. 3.1).
 *
 * Conventions for every entry point:
 *   - Every function returns a vecchia_status (0 = ok, < 0 = error).
 *   - Buffers are caller-owned; the library never frees or retains them past
 *     the call.  Array arguments may be host or device memory (the library asks
 *     the CUDA runtime which); results named "host" are always host memory.
 *   - Calls run on the context's stream and are synchronous at return.
 *   - sites are D x 2 row-major FP64 (x, y); indices are 0-based int32.
 *   - u are centred thresholds x - mu (Eq. int has mu; the ratio form of
 *     Eq. vecchia-cdf works with centred values).
 *   - Nothing here calls exit/abort; a CUDA error is returned as
 *     VECCHIA_ERR_CUDA and leaves the context usable when the device is.
 */
#ifndef VECCHIA_H
#define VECCHIA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VECCHIA_OK = 0,
    VECCHIA_ERR_ARG = -1,          /* invalid argument (size, kind, pointer, parameter) */
    VECCHIA_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    VECCHIA_ERR_NOMEM = -3,        /* device or host allocation failed */
    VECCHIA_ERR_NOT_PD = -4,       /* a covariance block is not positive definite */
    VECCHIA_ERR_NONFINITE = -5,    /* a term came out NaN/Inf or zero */
    VECCHIA_ERR_TIMEOUT = -6,      /* a bounded device wait ran out */
    VECCHIA_ERR_UNSUPPORTED = -7   /* valid request outside this build's limits (m > VECCHIA_MAX_M) */
} vecchia_status;

typedef enum {
    VECCHIA_ORDER_XY = 0,       /* by x, then y, then index */
    VECCHIA_ORDER_MAXMIN = 1,   /* exact maxmin on quantised coordinates */
    VECCHIA_ORDER_IDENTITY = 2  /* as given */
} vecchia_order_kind;

typedef enum {
    VECCHIA_COV_EXPONENTIAL = 0, /* variance * exp(-h / range)            (Sec. 3, Sec. 4.1) */
    VECCHIA_COV_MATERN = 1,      /* Rasmussen-Williams Matern, nu in {0.5, 1.5, 2.5} */
    VECCHIA_COV_ANISO_EXP = 2    /* variance * exp(-h / range), h the Mahalanobis distance of
                                    Sec. 4.1: Omega = (s_i - s_j)^T R(angle)^{-1} diag(1, aspect),
                                    h^2 = Omega Omega^T */
} vecchia_cov_kind;

/* Covariance C(s_i, s_j) of the spatial process; nugget adds to the diagonal
 * (0 for none).  nu is read for VECCHIA_COV_MATERN only; angle (radians) and
 * aspect (> 0) for VECCHIA_COV_ANISO_EXP only. */
typedef struct {
    int32_t kind;
    double variance;
    double range;
    double nu;
    double nugget;
    double angle;
    double aspect;
} vecchia_cov;

typedef enum {
    VECCHIA_FP64 = 0,  /* every step in FP64 */
    VECCHIA_MIXED = 1  /* FP64 covariance, Cholesky and sums; FP32 Genz integrand */
} vecchia_precision;

/* Largest conditioning-set size m of this build (terms of <= 64 variables). */
#define VECCHIA_MAX_M 63
/* Largest number of random shifts S per problem. */
#define VECCHIA_MAX_S 64

typedef struct vecchia_ctx vecchia_ctx;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns a
 * device scratch arena that grows on demand and is freed by vecchia_destroy. */
int vecchia_create(vecchia_ctx** ctx, int device, void* cuda_stream);
int vecchia_destroy(vecchia_ctx* ctx);
/* Change the stream later calls are issued on. */
int vecchia_set_stream(vecchia_ctx* ctx, void* cuda_stream);

/* Step a0 -- ordering of the sites (Sec. 2.1; Sec. 3.2 "ordering the
 * components by distance").  perm[new position] = old index (D int32, host or
 * device).  The caller applies perm to sites and u before the next calls.
 * With ctx = NULL both arrays are host memory and the ordering runs on the
 * host (MAXMIN: O(D^2) integer work over the host's cores).  With a context,
 * MAXMIN runs on the device (one persistent CTA: a tournament tree over the
 * distances to the chosen set, each pick scanning only the grid cells within
 * the current maximum distance), with the same result; XY with both arrays
 * on the device and D <= 8192 runs on the device (each site's rank by
 * counting the smaller keys); the other cases run on the host.  MAXMIN: first the site nearest the centre of the quantised
 * bounding box, then repeatedly the site farthest from the chosen ones, on
 * quantised coordinates, ties to the smaller index. */
int vecchia_order(vecchia_ctx* ctx, const double* sites, int64_t D, int kind, int32_t* perm);

/* Apply an ordering: sites_out[k] = sites[perm[k]] (D x 2) and, when u is not
 * NULL, u_out[k] = u[perm[k]].  All arrays device memory (a gather kernel on
 * the context's stream) or all host memory (ctx may then be NULL); outputs
 * must not alias inputs.  An index outside [0, D) is VECCHIA_ERR_ARG. */
int vecchia_apply_order(vecchia_ctx* ctx, const int32_t* perm, const double* sites, const double* u,
                        int64_t D, double* sites_out, double* u_out);

/* Step a1 -- conditioning sets (Sec. 2.1: the m nearest neighbours among the
 * previously ordered sites, |N_i| = min(m, i-1)).  On GPU: grid-bucketed
 * integer search on quantised coordinates, q = floor((x - xmin) * 2^30 /
 * extent); ties in squared distance go to the smaller index.  nbr is D x m
 * int32 (host or device), each row ascending, padded with -1.  0 <= m <= 63. */
int vecchia_neighbors(vecchia_ctx* ctx, const double* sites_ordered, int64_t D, int m, int32_t* nbr);

/* Steps a2-a7 -- the Vecchia log-CDF (Eq. vecchia-cdf) with Genz QMC on a
 * rank-1 Korobov lattice of N points (vecchia_lattice) and S random shifts
 * drawn from `seed` (vecchia_shifts); every term shares the same points
 * (common random numbers).  sites_ordered, u (D) and nbr (D x m, from
 * vecchia_neighbors) are host or device; log_p and std_err are host scalars:
 * the estimate of log P(X < u) and its delta-method standard error over the
 * S shifts.  N >= 1, 2 <= S <= VECCHIA_MAX_S, 0 <= m <= VECCHIA_MAX_M.
 * On VECCHIA_ERR_NOT_PD, vecchia_last_error_site() gives the ordered site. */
int vecchia_log_cdf(vecchia_ctx* ctx, const double* sites_ordered, int64_t D, const int32_t* nbr,
                    int m, vecchia_cov cov, const double* u, int64_t N, int S, uint64_t seed,
                    int precision, double* log_p, double* std_err);

/* As vecchia_log_cdf, and also returns the per-term pieces (any may be NULL;
 * each host or device): terms[i] = log mean_s num[i,s] - log mean_s den[i,s];
 * num, den (D x S): per-shift lattice means of the (q_i+1)- and q_i-dim CDFs. */
int vecchia_log_cdf_terms(vecchia_ctx* ctx, const double* sites_ordered, int64_t D,
                          const int32_t* nbr, int m, vecchia_cov cov, const double* u, int64_t N,
                          int S, uint64_t seed, int precision, double* log_p, double* std_err,
                          double* terms, double* num, double* den);

/* Steps a0-a7 in one call from unordered sites: the ordering (order_kind),
 * its application, the m-neighbour rows and the log-CDF, queued on the
 * context's stream with no host round trip in between (the XY ordering of
 * more than 8192 sites is the one host step); the same results as the four
 * calls in sequence.  sites (D x 2) and u (D) host or device, both of one
 * kind; perm_out (D, host or device) may be NULL, else it gets the ordering
 * (new position -> old index).  Other arguments as for vecchia_log_cdf. */
int vecchia_log_cdf_unordered(vecchia_ctx* ctx, const double* sites, const double* u, int64_t D, int order_kind,
                              int m, vecchia_cov cov, int64_t N, int S, uint64_t seed, int precision,
                              int32_t* perm_out, double* log_p, double* std_err);

/* One problem of a batch: the arguments of vecchia_log_cdf, or, with
 * group = p >= 1, of vecchia_grouped_log_cdf (nbr then holds the
 * ceil(D/p) x m conditioning rows of the groups and m is cmax). */
typedef struct {
    const double* sites;  /* D x 2, ordered */
    const int32_t* nbr;   /* D x m (group 0) or ceil(D/p) x m (group p) */
    const double* u;      /* D */
    int64_t D;
    int32_t m;
    int32_t S;
    int64_t N;
    uint64_t seed;
    vecchia_cov cov;
    int32_t group;        /* 0: one term per site (Eq. vecchia-cdf); p: joint groups of p sites */
    int32_t cond_max;     /* group p: the largest number of conditioning sites in any row (its
                           * leading non-negative entries), if known (0 = m).  Picks the kernel
                           * instantiation (the block size cond_max + p rather than m + p);
                           * a row with more entries makes its term fail with
                           * VECCHIA_ERR_ARG.  vecchia_grouped_log_cdf computes it. */
} vecchia_problem;

/* Many independent problems in one set of launches (the terms of every
 * problem form one work list; Sec. 3.1's parallelism across terms, extended
 * across problems).  The arrays of all problems must be of one kind (all host
 * or all device).  log_p, std_err, status are host arrays of n_probs; a
 * problem that fails gets its own status and NaN results; the call returns
 * VECCHIA_OK when the batch ran, even if some problems failed (a batch of
 * one problem returns that problem's status). */
int vecchia_log_cdf_batch(vecchia_ctx* ctx, const vecchia_problem* probs, int n_probs,
                          int precision, double* log_p, double* std_err, int32_t* status);

/* ---- joint groups and general conditioning sets (Sec. 3.2) ---------------
 * The ordered sites are split into groups k = 0 .. ceil(D/p) - 1 of p
 * consecutive sites [k p, min(k p + p, D)); group k is conditioned on a set
 * C_k of earlier sites (all < k p), and
 *   log P ~ sum_k [ log Phi(u_{C_k}, u_{G_k}) - log Phi(u_{C_k}) ]
 * with both CDFs from one Genz run on the block (C_k ascending, G_k): the
 * conditioning CDF is the leading |C_k|-dim block.  p = 1 with the nearest
 * neighbours is Eq. vecchia-cdf. */
typedef enum {
    VECCHIA_COND_NEAREST = 0, /* union of the m nearest earlier sites of each member (first method) */
    VECCHIA_COND_RANDOM = 1   /* m sites drawn uniformly without replacement among the earlier ones
                                 (second method; the third is m = p m') */
} vecchia_cond_method;

/* Conditioning sets of the groups: cond (ceil(D/p) x cmax int32, rows
 * ascending, -1 padded) and count (ceil(D/p) int32, may be NULL), both host or
 * both device.  NEAREST: quantised squared distance, ties to the smaller
 * index, as vecchia_neighbors (p = 1 gives its rows); VECCHIA_ERR_ARG when a
 * union has more than cmax sites (cmax >= p m always suffices).  RANDOM: a
 * uniform subset of min(m, k p) sites before group k by Floyd's algorithm,
 * draw r of group k the integer floor(w (j + 1) / 2^32), w the first word of
 * Philox4x32-10 with key (seed lo, seed hi) and counter (k lo, r, 0x52C5,
 * k hi); m <= cmax.  sites_ordered: D x 2 (same memory kind as cond);
 * 1 <= p, 0 <= m <= VECCHIA_MAX_M, cmax + p <= VECCHIA_MAX_M + 1. */
int vecchia_group_conditioning(vecchia_ctx* ctx, const double* sites_ordered, int64_t D, int p, int m,
                               int method, uint64_t seed, int cmax, int32_t* cond, int32_t* count);

/* The grouped log-CDF: as vecchia_log_cdf with the conditioning rows cond
 * (ceil(D/p) x cmax, from vecchia_group_conditioning or the caller: rows
 * ascending, entries < k p, -1 padded after the last).  Terms have up to
 * cmax + p <= VECCHIA_MAX_M + 1 variables.  On VECCHIA_ERR_NOT_PD or a bad
 * row, vecchia_last_error_site() gives the group index.  The call first finds
 * the longest row (a reduction on the device when cond is device memory) and
 * evaluates with the kernel sized for it (vecchia_problem.cond_max). */
int vecchia_grouped_log_cdf(vecchia_ctx* ctx, const double* sites_ordered, int64_t D, int p,
                            const int32_t* cond, int cmax, vecchia_cov cov, const double* u, int64_t N,
                            int S, uint64_t seed, int precision, double* log_p, double* std_err);

/* ---- building blocks for schedulers (continuous batching) ----------------
 * The result slot of a problem, in device memory; the layout the library
 * writes.  status is a vecchia_status; bad_site the first failing term (the
 * ordered site, or the group index of a grouped problem)
 * (INT64_MAX when none). */
typedef struct {
    double log_p;
    double std_err;
    int64_t bad_site;
    int32_t status;
    int32_t reserved;
} vecchia_result;

/* A range of terms of one problem (sites, or groups when prob.group > 0):
 * the Genz partial means of terms site_begin .. site_begin + site_count - 1
 * (all shifts) are written into num/den (terms x S, device), failures into
 * *result (device).  All arrays are
 * device memory that stays valid until the work has run on the stream. */
typedef struct {
    vecchia_problem prob;
    double* num;
    double* den;
    vecchia_result* result;
    int64_t site_begin;
    int64_t site_count;
} vecchia_segment;

/* vecchia_neighbors for device arrays without waiting: queued on the
 * context's stream (stream-ordered with the other calls) and returning at
 * once.  sites_ordered and nbr must be device memory. */
int vecchia_neighbors_async(vecchia_ctx* ctx, const double* sites_ordered, int64_t D, int m,
                            int32_t* nbr);
/* Set n result slots to {0, 0, INT64_MAX, VECCHIA_OK} (stream-ordered). */
int vecchia_result_init(vecchia_ctx* ctx, vecchia_result* results, int n);
/* Steps a2-a6 for the given site segments of any problems, in one set of
 * launches on the context's stream; returns without waiting (stream-ordered
 * with earlier and later calls on the context).  Segments of different
 * problems, different m, N, S and covariances mix freely; a site's partial
 * means do not depend on which segments it was launched with.  Invalid
 * segments make the whole call VECCHIA_ERR_ARG before anything is queued. */
int vecchia_partials_async(vecchia_ctx* ctx, const vecchia_segment* segs, int n_segs, int precision);
/* Step a7 for whole problems whose partials are complete (site ranges are
 * ignored): writes log_p, std_err (and VECCHIA_ERR_NONFINITE) into each
 * problem's result slot; stream-ordered, returns without waiting. */
int vecchia_reduce_async(vecchia_ctx* ctx, const vecchia_segment* probs, int n_probs);

/* A plan: a batch prepared once and replayed, for callers that evaluate the
 * same sites and neighbour lists many times with new covariance parameters or
 * QMC seeds (a likelihood optimiser, Sec. 4.1, calls the log-CDF at every
 * parameter value).  vecchia_plan_create validates the batch, keeps its inputs
 * resident (host arrays are copied once; device arrays are read in place and
 * must stay valid and unchanged while the plan lives), allocates the plan's
 * own device and pinned host buffers, runs the batch once and captures its
 * whole device sequence (parameter upload, shift tables, Genz kernels, the
 * re-evaluation pass, log-sum, result download) as one CUDA graph.
 * vecchia_plan_run replays the graph with new seeds and/or covariances
 * (arrays of n_probs, either may be NULL to keep the previous ones) on the
 * plan's own stream, ordered after work already queued on the context's
 * stream, and returns host results like vecchia_log_cdf_batch.  Results are
 * identical to vecchia_log_cdf_batch on the same inputs. */
typedef struct vecchia_plan vecchia_plan;
int vecchia_plan_create(vecchia_ctx* ctx, const vecchia_problem* probs, int n_probs, int precision,
                        vecchia_plan** plan, int32_t* status);
int vecchia_plan_run(vecchia_plan* plan, const uint64_t* seeds, const vecchia_cov* covs, double* log_p,
                     double* std_err, int32_t* status);
int vecchia_plan_destroy(vecchia_plan* plan);

/* The scale-mixture CDF of Sec. 4 (Eq. model01-model03): X = R W with W the
 * Gaussian process of `cov` and R independent with
 *   F_R(r) = 1 - exp(-gamma (r^beta - 1) / beta),  r >= 1, beta > 0,
 *   F_R(r) = 1 - r^(-gamma)                            (beta = 0, the limit),
 * G(x) = P(X < x) = int Phi_D(x / r; Sigma) dF_R(r).  With v = F_R(r) the
 * integral is over [0, 1]; the substitution v = 1 - (1 - t)^4 removes the
 * singularity of F_R^{-1} at v = 1, and an n_nodes-point Gauss-Legendre rule
 * in t (quadrature error of log G about 1e-6 or less at 16 nodes for
 * beta >= 0.2, gamma >= 1, |x| <= 4 in one dimension) together with
 * Phi_D(x / r; Sigma) = Phi_D(x; r^2 Sigma) turn it into n_nodes Vecchia
 * log-CDFs on the same sites and neighbour lists with the covariance scaled by
 * r^2, evaluated as one batch (common random numbers across nodes).
 * log_g = log sum_q w_q P_q; std_err bounds the QMC error of log_g by full
 * correlation of the nodes' errors.  beta >= 0, gamma > 0, 1 <= n_nodes <= 256;
 * other arguments as for vecchia_log_cdf (x are the centred thresholds). */
int vecchia_mixture_log_cdf(vecchia_ctx* ctx, const double* sites_ordered, int64_t D,
                            const int32_t* nbr, int m, vecchia_cov cov, const double* x, int64_t N,
                            int S, uint64_t seed, double beta, double gamma, int n_nodes,
                            int precision, double* log_g, double* std_err);

/* The full D-dimensional Genz estimate of P(X < u) (Sec. 2.2, Sec. 3) on the
 * same rank-1 lattice (dimension D - 1) and shifts as the Vecchia terms: the
 * m = D - 1 limit of Eq. (vecchia-cdf), which telescopes (Eq.
 * cascading-conditional-cdf) -- the estimate the approximation is compared
 * with.  Covariance and Cholesky in FP64 (blocked, 32 columns a block; FP64
 * path: each entry of the factor takes its terms in ascending order with fma,
 * then the pivot division; mixed path: the same, except that the trailing
 * update of each block column runs on the tensor cores from bf16 digit slices
 * of the block column at FP64 accuracy, see vecchia_full_cholesky); the
 * recursion over all D variables in the precision requested (mixed: FP32
 * integrand, conditional means on the tensor cores from TF32 hi/lo splits of
 * the FP32 operands -- FP32-level accuracy --, FP64 running product and
 * sums).  log_p = log of the mean over shifts of the lattice means; rel_se =
 * their standard error over the mean.  Arrays host or device (both of one
 * kind); device memory grows as about 16 D^2 + 9.2 (mixed) or 8 (FP64) D S N
 * bytes.  D <= VECCHIA_FULL_MAX_D.  A non-positive pivot gives
 * VECCHIA_ERR_NOT_PD with its site in vecchia_last_error_site();
 * VECCHIA_ERR_TIMEOUT means a bounded device wait of the mixed recursion ran
 * out (2 s without progress). */
#define VECCHIA_FULL_MAX_D 32768
int vecchia_full_genz(vecchia_ctx* ctx, const double* sites_ordered, int64_t D, vecchia_cov cov,
                      const double* u, int64_t N, int S, uint64_t seed, int precision, double* log_p,
                      double* rel_se);

/* Diagnostic: the covariance of D sites (D x 2, host or device) and its
 * Cholesky factor as vecchia_full_genz computes them, into L (D x D row-major,
 * host or device, caller-owned): the lower triangle gets the factor, the
 * strict upper triangle zeros.  precision VECCHIA_FP64: the FP64 blocked
 * factor; VECCHIA_MIXED: each block column's trailing update on the tensor
 * cores -- its rows written as 2^e times seven balanced base-256 digits
 * (bf16), the digit products of each significance summed exactly in FP32
 * accumulators, recombined in 64-bit integers and subtracted with one FP64
 * rounding (error below a few 2^-53 of sum_t |L_rt L_ct|).  D <=
 * VECCHIA_FULL_MAX_D.  VECCHIA_ERR_NOT_PD with the failing row in
 * vecchia_last_error_site(); VECCHIA_ERR_TIMEOUT if a bounded device wait of
 * the tensor-core update ran out. */
int vecchia_full_cholesky(vecchia_ctx* ctx, const double* sites_ordered, int64_t D, vecchia_cov cov,
                          int precision, double* L);

/* The censored likelihood G_I of Sec. 4 (Eq. model05) for one replicate:
 * the nc censored values (sites_c ordered, x_c, neighbour rows nbr nc x m
 * among them) are below the threshold, the ni observed ones (sites_i, x_i)
 * above it.  With Sigma_II = L L^T over the observed sites,
 *   G_I = int Phi_nc{(x_c - mu)/r; Sigma_{c|I}} phi_ni(x_I / r; Sigma_II) r^-ni dF_R(r),
 *   mu = Sigma_cI Sigma_II^-1 x_I,  Sigma_{c|I} = Sigma_cc - Sigma_cI Sigma_II^-1 Sigma_Ic,
 * Phi_nc by Eq. (vecchia-cdf) on the censored sites with the conditional
 * covariance (each block entry minus V_a . V_b, V = L^-1 Sigma_Ic, on the
 * device), phi in closed form, and the integral by the rule of
 * vecchia_mixture_log_cdf (n_nodes >= 1; beta, gamma of Eq. model02);
 * n_nodes = 0 takes R = 1, the Gaussian censored likelihood.  ni = 0 is
 * vecchia_mixture_log_cdf (or vecchia_log_cdf); nc = 0 the density alone.
 * Arrays host or device, all of one kind; 1 <= nc + ni, ni <=
 * VECCHIA_CENSOR_MAX_OBS.  A non-positive pivot of Sigma_II gives
 * VECCHIA_ERR_NOT_PD with the observed site's index in
 * vecchia_last_error_site(). */
#define VECCHIA_CENSOR_MAX_OBS 4096
int vecchia_censored_log_cdf(vecchia_ctx* ctx, const double* sites_c, int64_t nc, const int32_t* nbr, int m,
                             const double* sites_i, int64_t ni, vecchia_cov cov, const double* x_c,
                             const double* x_i, int64_t N, int S, uint64_t seed, double beta, double gamma,
                             int n_nodes, int precision, double* log_g, double* std_err);

/* Korobov generating vector g[j] = a^j mod N, j < dim (host array): a in
 * [2, N/2], gcd(a, N) = 1, minimising the weighted P2 criterion over 30
 * dimensions with weights 1/j^2 (ties: smaller a).  N < 4 gives a = 1. */
int vecchia_lattice(int64_t N, int dim, uint32_t* g);

/* The random shifts of `seed` (host array S x dim): 53-bit uniforms from
 * Philox4x32-10, key (seed lo, seed hi), counter (s, j, 0x51A7, 0). */
int vecchia_shifts(uint64_t seed, int S, int dim, double* delta);

/* Launch tile of the fused Genz kernel for one precision and block bucket
 * (bucket b holds problems whose largest term has d <= 9, 13, 17, 21, 25,
 * 29, 32, 48, 64 variables for b = 0..8 -- d = m + 1, or m + p for groups of
 * p; -1 = all): warps per CTA (1..16; at most 8 above 32 variables), points
 * per lane per pass (1 or 2; FP64 and blocks above 32 variables use 1),
 * lattice slices per shift spread over a CTA's warps (>= 1), shift groups per
 * term spread over CTAs (1..VECCHIA_MAX_S).  Tiles change only the launch
 * shape; results are identical up to the order of the final FP64 sums. */
int vecchia_set_tile(vecchia_ctx* ctx, int precision, int bucket, int warps, int points,
                     int slices, int groups);
/* Back to the built-in tile rule for every precision and bucket. */
int vecchia_reset_tiles(vecchia_ctx* ctx);
/* Record CUDA events around the Genz launches of each call (0 = off); for
 * vecchia_full_genz, around its recursion kernel alone. */
int vecchia_set_timing(vecchia_ctx* ctx, int enable);
/* Milliseconds between those events in the last call with timing on. */
int vecchia_genz_time_ms(const vecchia_ctx* ctx, double* ms);

/* Bounded device waits of vecchia_full_genz's tensor-core recursion (mixed
 * precision; the paper has no counterpart: this is how the library reports a
 * stalled kernel instead of hanging).  Its point warps wait on mbarriers for
 * the accumulators and its copy lane for their progress; a wait with no
 * progress for limit_ns (0 = the built-in 2 s; values above it are clamped
 * to it) makes the kernel record a timeout, wait (with the full 2 s limit)
 * for every copy and MMA it has issued, free its tensor memory and return,
 * and the call then returns VECCHIA_ERR_TIMEOUT.  withhold != 0 is for tests
 * of that path only: the copy lane issues no copy and no MMA, so the first
 * accumulator wait runs out with nothing in flight.  The setting stays on the
 * context until changed; (0, 0) restores the default. */
int vecchia_set_full_genz_wait(vecchia_ctx* ctx, uint64_t limit_ns, int withhold);

/* Diagnostic: the FP32 special functions of the mixed path on n values (x and
 * out device arrays of float): which = 0: Phi(x); 1: 1 - Phi(x); 2: log2 Phi(x)
 * for x < -9 (NaN otherwise); 3: Phi^{-1}(x), x in (0, 1); 4: Phi^{-1}(2^x) for
 * x < -64; the forms of the fast mixed step: 5: Phi(x / k) and 6: 1 - Phi(x / k),
 * k = sqrt(log2(e) / 2) (its recursion carries k z); 7: Phi^{-1}(x) from 16 x
 * and 16 (1 - x).  These are the maps of Genz's separation of variables
 * (Sec. 2.2) in the precision the mixed path evaluates them. */
int vecchia_eval_special(vecchia_ctx* ctx, int which, const float* x, int64_t n, float* out);

/* Diagnostic: the FP64 special functions of the FP64 path on n values (x and
 * out device arrays of double): which = 0: Phi(x); 1: 1 - Phi(x) (from the
 * tail); 2: Phi^{-1}(x) given p = x, q = 1 - x; 3: Phi^{-1}(1 - x) given q = x
 * (the upper tail, to full precision).  The same maps (Sec. 2.2) in FP64. */
int vecchia_eval_special64(vecchia_ctx* ctx, int which, const double* x, int64_t n, double* out);

/* Size of the fixed device array that vecchia_log_cdf_noalloc uses as scratch. */
#define VECCHIA_NOALLOC_SCRATCH_BYTES (32u << 20)

/* vecchia_log_cdf for callers that cannot allocate memory (the paper has no
 * counterpart; this is a deployment variant of the same kernels).  Programs
 * whose allocator owns the whole device and forbids foreign cudaMalloc calls,
 * code that must run within a fixed memory budget (no allocation after
 * start-up), and hosts that keep no vecchia_ctx cannot use the context's
 * scratch arena.  This entry point keeps
 * all of its scratch in one file-scope device array of
 * VECCHIA_NOALLOC_SCRATCH_BYTES (32 MiB, held by every GPU that loads the
 * library until the process exits) and calls no allocating routine: no
 * cudaMalloc, cudaFree or cudaMallocHost, and no context is needed.
 *   device, cuda_stream: where to run (stream NULL = legacy default stream);
 *   the stream must belong to `device`.  The call makes `device` current
 *   while it runs and restores the calling thread's current device before it
 *   returns.
 *   sites_ordered (D x 2), nbr (D x m), u (D): device memory on `device`
 *   (memory of another GPU, or host memory, gives VECCHIA_ERR_ARG), as for
 *   vecchia_log_cdf; log_p, std_err: host scalars.
 * A problem whose scratch (about 16 D S + 16 D bytes, plus 8 D per shift group
 * on the mixed path) exceeds the array returns VECCHIA_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address (once per
 * device, under a lock); make that first call before any stream capture.
 * Every call uploads its parameters from the host and synchronises
 * cuda_stream before it returns.
 * Every call shares the array and clears what must start at zero; calls
 * whose work overlaps on the GPU (other streams or host threads on the same
 * device) race on it and must be serialised by the caller.  Results equal
 * vecchia_log_cdf's with the built-in tile bit for bit. */
int vecchia_log_cdf_noalloc(int device, void* cuda_stream, const double* sites_ordered, int64_t D,
                            const int32_t* nbr, int m, vecchia_cov cov, const double* u, int64_t N,
                            int S, uint64_t seed, int precision, double* log_p, double* std_err);

/* Ordered index of the site whose block failed in the last call (or -1). */
int64_t vecchia_last_error_site(const vecchia_ctx* ctx);

/* Static description of a status code. */
const char* vecchia_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* VECCHIA_H */
