/*
 * vref.h -- the oracle: a plain, slow FP64 CPU restatement of the Vecchia
 * approximation to a Gaussian CDF (Nascimento & Shaby, arXiv 2007.15195).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no source, header, table or constant generator with the CUDA library under
 * paper_2007_15195_gb300/; the two meet only through seeded inputs.
 *
 * Every routine is written to be checked against the paper by eye:
 *   - Sec. 2.2, Eq. (vecchia-cdf): F(x) ~ Phi(x_1) prod_{i>=2}
 *       Phi(x_{i,N_i}) / Phi(x_{N_i}),  |N_i| = min(m, i-1);
 *   - Sec. 2.1: N_i = the m nearest previously ordered sites;
 *   - Sec. 2.2 / Sec. 3: each low-dimensional CDF by Genz's
 *     separation-of-variables quasi-Monte Carlo (randomly shifted lattice);
 *   - Sec. 3.1: every term on the log scale, then one sum.
 * Readings of what the paper leaves open (lattice, shifts, tie-breaks,
 * standard error) are stated beside the routine that takes them.
 *
 * Status codes: 0 ok, -1 bad argument, -4 covariance block not positive
 * definite.  Arrays are caller-owned, row-major, host memory.
 */
#ifndef VREF_H
#define VREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { VREF_OK = 0, VREF_ERR_ARG = -1, VREF_ERR_NOT_PD = -4 };
enum { VREF_COV_EXPONENTIAL = 0, VREF_COV_MATERN = 1, VREF_COV_ANISO_EXP = 2 };

/* A covariance function: exponential sigma^2 exp(-h/rho); Matern (nu in
 * {0.5, 1.5, 2.5}); or the anisotropic exponential of Sec. 4.1, whose h is
 * the Mahalanobis distance with rotation `angle` and aspect ratio `aspect`.
 * The nugget is added on the diagonal. */
typedef struct {
    int kind;
    double variance, range, nu, nugget, angle, aspect;
} vref_cov_t;
enum { VREF_ORDER_XY = 0, VREF_ORDER_MAXMIN = 1, VREF_ORDER_IDENTITY = 2 };

/* ---- univariate normal ------------------------------------------------- */
/* Phi(x) = erfc(-x/sqrt 2)/2 (libm erfc). */
double vref_Phi(double x);
/* Phi(-|x|): the smaller tail, to full relative precision. */
double vref_Phi_tail(double x);
/* Inverse of Phi on (0, 1/2]: Wichura's AS241 (PPND16, Applied Statistics
 * 37, 1988) followed by one Halley step on erfc.  Returns a value <= 0. */
double vref_Phiinv_lower(double r);
/* Phi^{-1}(p) with q = 1 - p supplied separately (both >= 0, p + q ~ 1):
 * evaluates from the smaller of p and q, each clamped below at 2^-1000. */
double vref_Phiinv_pq(double p, double q);
/* Phi^{-1}(p) for p in (0,1) (convenience: q = 1 - p). */
double vref_Phiinv(double p);

/* ---- randomisation: Philox4x32-10 and the shifts ------------------------- */
/* Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11: the 10-round Philox-4x32 bijection. */
void vref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* delta[s*dim + j] = 53-bit uniform in [0,1) from Philox with
 * key = (seed lo32, seed hi32), counter = (s, j, 0x51A7, 0):
 * ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53. */
int vref_shifts(uint64_t seed, int S, int dim, double* delta);

/* ---- rank-1 Korobov lattice -------------------------------------------- */
/* Weighted P2 criterion of the Korobov vector g_j = a^j mod N, j < dim,
 * weights gamma_j = 1/(j+1)^2:
 *   P2 = -1 + (1/N) sum_k prod_j (1 + gamma_j 2 pi^2 B2({k g_j / N})),
 *   B2(x) = x^2 - x + 1/6. */
double vref_p2(int64_t N, int64_t a, int dim);
/* a in [2, N/2] with gcd(a, N) = 1 minimising P2 over dim 30 (ties: smaller
 * a).  N < 4 gives a = 1. */
int64_t vref_korobov_a(int64_t N);
/* g[j] = a^j mod N, j < dim, a = vref_korobov_a(N). */
int vref_lattice(int64_t N, int dim, uint32_t* g);

/* ---- covariance and Cholesky --------------------------------------------- */
/* Isotropic covariance at distance h:
 *   exponential: var exp(-h/range)                       (Sec. 3)
 *   Matern nu=0.5: same; nu=1.5: var (1+sqrt3 h/r) exp(-sqrt3 h/r);
 *   nu=2.5: var (1+sqrt5 h/r+5h^2/(3r^2)) exp(-sqrt5 h/r)
 *   (Rasmussen-Williams form).  Unsupported nu returns NaN. */
double vref_cov(int kind, double variance, double range, double nu, double h);
/* Dense covariance matrix of `n` sites (n x 2), nugget added to the diagonal. */
int vref_cov_matrix(const double* sites, int64_t n, int kind, double variance, double range,
                    double nu, double nugget, double* Sigma);
/* Row-by-row Cholesky (Banachiewicz): L lower, row-major d x d, inner sums
 * in ascending index with explicit fma.  A pivot <= 0 or NaN -> NOT_PD. */
int vref_cholesky(int d, const double* A, double* L);

/* ---- ordering and neighbours (integer work on quantised coordinates) ----- */
/* q[2i], q[2i+1] = floor((x - xmin) * c), c = 2^30 / max(xmax-xmin, ymax-ymin)
 * (all zeros if the extent is 0).  Round-to-nearest, no contraction. */
int vref_quantize(const double* sites, int64_t D, int64_t* q);
/* perm[new position] = old index.  XY: stable sort by (x, y, index).
 * MAXMIN: first the site nearest the centre of the quantised bounding box,
 * then repeatedly the site whose minimum quantised squared distance to the
 * chosen set is largest (ties: smaller index). IDENTITY: 0..D-1. */
int vref_order(const double* sites, int64_t D, int kind, int32_t* perm);
/* nbr[i*m + r]: the min(m, i) sites j < i nearest to i by (quantised d^2, j),
 * listed ascending in j, padded with -1.  Sites are already ordered. */
int vref_neighbors(const double* sites, int64_t D, int m, int32_t* nbr);
/* The same for one site i (out has m entries). */
int vref_neighbors_of(const double* sites, int64_t D, int64_t i, int m, int32_t* out);

/* ---- Genz separation-of-variables QMC ------------------------------------ */
/* For the d-dimensional N(0, Sigma) CDF at u (Sigma d x d row-major):
 * per shift s, num[s] = (1/N) sum_k f_d(k,s) and den[s] = (1/N) sum_k
 * f_{d-1}(k,s), where f_t is the product of the first t conditional
 * probabilities of Genz's recursion at the tent-transformed shifted lattice
 * point x_{k,j} = frac((k g_j mod N)/N + delta[s*dim + j]).  d = 1 gives
 * num[s] = Phi(u_1/sqrt(Sigma_11)), den[s] = 1.  dim >= d - 1. */
int vref_genz_sums(int d, const double* Sigma, const double* u, int64_t N, int S,
                   const uint32_t* g, const double* delta, int dim, double* num, double* den);
/* Full Genz estimate of P(X < u) with the lattice for N and shifts for seed:
 * p = mean over shifts of num[s]; rel_se = sd over shifts / (p sqrt S). */
int vref_genz_cdf(int d, const double* Sigma, const double* u, int64_t N, int S, uint64_t seed,
                  double* p, double* rel_se);

/* ---- the Vecchia log-CDF (Eq. vecchia-cdf) -------------------------------- */
/* Per-site partial sums for the sites listed in `sites_idx` (n_idx of them;
 * NULL = all D): num[r*S + s], den[r*S + s] for the (q+1)-dim CDF of the
 * block (N_i ascending, i) and the q-dim CDF of N_i, q = min(m, i). */
int vref_vecchia_partials(const double* sites, int64_t D, const int32_t* nbr, int m, int cov_kind,
                          double variance, double range, double nu, double nugget, const double* u,
                          int64_t N, int S, uint64_t seed, const int64_t* sites_idx, int64_t n_idx,
                          double* num, double* den, int64_t* bad_site);
/* Reduction over sites: T_i = log mean_s num - log mean_s den; log_p = sum_i
 * T_i (ascending i); l_s = sum_i (num_is/numbar_i - den_is/denbar_i);
 * se = sqrt(sum_s l_s^2 / (S (S-1))).  terms may be NULL. */
int vref_vecchia_reduce(int64_t D, int S, const double* num, const double* den, double* log_p,
                        double* se, double* terms);
/* Partials + reduction for the whole problem. */
int vref_log_cdf(const double* sites, int64_t D, const int32_t* nbr, int m, int cov_kind,
                 double variance, double range, double nu, double nugget, const double* u,
                 int64_t N, int S, uint64_t seed, double* log_p, double* se, double* terms,
                 int64_t* bad_site);
/* log of the full D-dimensional Genz estimate on the same lattice and shifts
 * (the m = D-1 limit of the telescoping product, Eq. cascading-conditional-cdf). */
int vref_full_genz(const double* sites, int64_t D, int cov_kind, double variance, double range,
                   double nu, double nugget, const double* u, int64_t N, int S, uint64_t seed,
                   double* log_p, double* se);

/* Number of OpenMP threads the partials loop uses. */
int vref_num_threads(void);

/* ---- general terms: joint groups and conditioning sets (Sec. 3.2) ------- */
/* As vref_genz_sums for the d-dim block, except that den[s] is the sample mean
 * of the product of the first c conditional probabilities: the c-dim CDF of
 * the leading block (0 <= c <= d-1; c = 0 gives den = 1). */
int vref_genz_sums_c(int d, int c, const double* Sigma, const double* u, int64_t N, int S,
                     const uint32_t* g, const double* delta, int dim, double* num, double* den);
/* Groups k = 0..ceil(D/p)-1 of p consecutive ordered sites [k p, k p + p).
 * Nearest conditioning (Sec. 3.2, first method): the union of the min(m, k p)
 * nearest sites before the group of each group member, ascending; cond is
 * G x cmax (-1 padded), count[k] its length; ERR_ARG if a union exceeds cmax. */
int vref_group_cond_nearest(const double* sites, int64_t D, int p, int m, int cmax, int32_t* cond,
                            int32_t* count);
/* Random conditioning (Sec. 3.2, second and third methods, kk = m or p m): a
 * uniform subset of min(kk, k p) sites before group k by Floyd's algorithm,
 * draw r of group k an integer in [0, j] from Philox4x32-10 with key = seed,
 * counter = (k lo32, r, 0x52C5, k hi32): floor(word0 (j + 1) / 2^32). */
int vref_group_cond_random(int64_t D, int p, int kk, uint64_t seed, int cmax, int32_t* cond,
                           int32_t* count);
/* Mahalanobis distance of Sec. 4.1 for the offset (dx, dy). */
double vref_aniso_h(double dx, double dy, double angle, double aspect);
int vref_cov_matrix_t(const double* sites, int64_t n, const vref_cov_t* cv, double* Sigma);
/* Per group k: the joint CDF of (C_k ascending, group sites) and the CDF of
 * C_k from one Genz run (num, den G x S); terms on the log scale as in
 * vref_vecchia_reduce.  Lattice and shifts for dim = cmax + p - 1. */
int vref_grouped_partials(const double* sites, int64_t D, int p, const int32_t* cond, int cmax,
                          const vref_cov_t* cv, const double* u, int64_t N, int S, uint64_t seed,
                          double* num, double* den, int64_t* bad_term);
int vref_grouped_log_cdf(const double* sites, int64_t D, int p, const int32_t* cond, int cmax,
                         const vref_cov_t* cv, const double* u, int64_t N, int S, uint64_t seed,
                         double* log_p, double* se, double* terms, int64_t* bad_term);

#ifdef __cplusplus
}
#endif
#endif
