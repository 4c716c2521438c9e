/*
 * vref.c -- the oracle (test infrastructure only; see vref.h).
 *
 * Plain FP64 C11, libm for exp/log/erfc/sqrt, OpenMP only across
 * independent Vecchia terms (Sec. 3.1: the terms are independent and are
 * computed in parallel, then summed).  Compiled with -ffp-contract=off so
 * that every product and sum is rounded exactly as written.
 */
#include "vref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VREF_PI 3.14159265358979323846
#define VREF_SQRT1_2 0.70710678118654752440
#define VREF_SQRT2PI 2.50662827463100050242

/* ======================================================================== */
/* Univariate normal CDF and its inverse                                     */
/* ======================================================================== */

double vref_Phi(double x) { return 0.5 * erfc(-x * VREF_SQRT1_2); }

double vref_Phi_tail(double x) { return 0.5 * erfc(fabs(x) * VREF_SQRT1_2); }

/* AS241 (Wichura 1988), algorithm PPND16: rational approximations to the
 * normal quantile in three regions of p, about 16 significant digits. */
static double as241_ppnd16(double p) {
    const double q = p - 0.5;
    if (fabs(q) <= 0.425) {
        const double r = 0.180625 - q * q;
        const double num =
            ((((((2.5090809287301226727e+3 * r + 3.3430575583588128105e+4) * r +
                 6.7265770927008700853e+4) * r + 4.5921953931549871457e+4) * r +
               1.3731693765509461125e+4) * r + 1.9715909503065514427e+3) * r +
             1.3314166789178437745e+2) * r + 3.3871328727963666080e+0;
        const double den =
            ((((((5.2264952788528545610e+3 * r + 2.8729085735721942674e+4) * r +
                 3.9307895800092710610e+4) * r + 2.1213794301586595867e+4) * r +
               5.3941960214247511077e+3) * r + 6.8718700749205790830e+2) * r +
             4.2313330701600911252e+1) * r + 1.0;
        return q * num / den;
    }
    double r = (q < 0.0) ? p : 1.0 - p;
    r = sqrt(-log(r));
    double val;
    if (r <= 5.0) {
        r -= 1.6;
        const double num =
            ((((((7.74545014278341407640e-4 * r + 2.27238449892691845833e-2) * r +
                 2.41780725177450611770e-1) * r + 1.27045825245236838258e+0) * r +
               3.64784832476320460504e+0) * r + 5.76949722146069140550e+0) * r +
             4.63033784615654529590e+0) * r + 1.42343711074968357734e+0;
        const double den =
            ((((((1.05075007164441684324e-9 * r + 5.47593808499534494600e-4) * r +
                 1.51986665636164571966e-2) * r + 1.48103976427480074590e-1) * r +
               6.89767334985100004550e-1) * r + 1.67638483018380384940e+0) * r +
             2.05319162663775882187e+0) * r + 1.0;
        val = num / den;
    } else {
        r -= 5.0;
        const double num =
            ((((((2.01033439929228813265e-7 * r + 2.71155556874348757815e-5) * r +
                 1.24266094738807843860e-3) * r + 2.65321895265761230930e-2) * r +
               2.96560571828504891230e-1) * r + 1.78482653991729133580e+0) * r +
             5.46378491116411436990e+0) * r + 6.65790464350110377720e+0;
        const double den =
            ((((((2.04426310338993978564e-15 * r + 1.42151175831644588870e-7) * r +
                 1.84631831751005468180e-5) * r + 7.86869131145613259100e-4) * r +
               1.48753612908506148525e-2) * r + 1.36929880922735805310e-1) * r +
             5.99832206555887937690e-1) * r + 1.0;
        val = num / den;
    }
    return (q < 0.0) ? -val : val;
}

double vref_Phiinv_lower(double r) {
    double x = as241_ppnd16(r);
    /* One Halley step for Phi(x) = r, with the residual taken relative to r
     * so that it stays a normal number deep in the tail:
     *   u = (Phi(x) - r)/phi(x) = (Phi(x)/r - 1) * r sqrt(2 pi) exp(x^2/2),
     *   x <- x - u / (1 + x u / 2). */
    const double rel = vref_Phi(x) / r - 1.0;
    const double u = rel * (r * VREF_SQRT2PI * exp(0.5 * x * x));
    x = x - u / (1.0 + 0.5 * x * u);
    return x;
}

#define VREF_P_FLOOR 9.3326361850321887899e-302 /* 2^-1000 */

double vref_Phiinv_pq(double p, double q) {
    const double pc = (p < VREF_P_FLOOR) ? VREF_P_FLOOR : p;
    const double qc = (q < VREF_P_FLOOR) ? VREF_P_FLOOR : q;
    if (pc <= qc) return vref_Phiinv_lower(pc);
    return -vref_Phiinv_lower(qc);
}

double vref_Phiinv(double p) { return vref_Phiinv_pq(p, 1.0 - p); }

/* ======================================================================== */
/* Philox4x32-10 and the random shifts                                       */
/* ======================================================================== */

void vref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* Weyl key schedule */
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

int vref_shifts(uint64_t seed, int S, int dim, double* delta) {
    if (S < 0 || dim < 0 || (S * dim > 0 && !delta)) return VREF_ERR_ARG;
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int s = 0; s < S; ++s) {
        for (int j = 0; j < dim; ++j) {
            const uint32_t ctr[4] = {(uint32_t)s, (uint32_t)j, 0x51A7u, 0u};
            uint32_t w[4];
            vref_philox4x32_10(ctr, key, w);
            const double hi = (double)(w[0] >> 5); /* 27 bits */
            const double lo = (double)(w[1] >> 6); /* 26 bits */
            delta[(int64_t)s * dim + j] = (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0);
        }
    }
    return VREF_OK;
}

/* ======================================================================== */
/* Korobov lattice                                                           */
/* ======================================================================== */

#define VREF_P2_DIM 30

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* B2(r/N) for r = 0..N-1; the same expression for every caller. */
static double* b2_table(int64_t N) {
    double* b = (double*)malloc(sizeof(double) * (size_t)N);
    if (!b) return NULL;
    for (int64_t r = 0; r < N; ++r) {
        const double x = (double)r / (double)N;
        b[r] = (x * x - x) + (1.0 / 6.0);
    }
    return b;
}

static double p2_with_table(int64_t N, int64_t a, int dim, const double* b2) {
    int64_t g[256];
    int64_t r[256];
    double c[256];
    if (dim > 256) dim = 256;
    const double two_pi_sq = 2.0 * VREF_PI * VREF_PI;
    int64_t gj = 1 % N;
    for (int j = 0; j < dim; ++j) {
        g[j] = gj;
        gj = (gj * a) % N;
        r[j] = 0;
        c[j] = two_pi_sq / (double)((j + 1) * (j + 1));
    }
    double acc = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        double prod = 1.0;
        for (int j = 0; j < dim; ++j) prod *= (1.0 + c[j] * b2[r[j]]);
        acc += prod;
        for (int j = 0; j < dim; ++j) { /* r_j = (k+1) g_j mod N */
            r[j] += g[j];
            if (r[j] >= N) r[j] -= N;
        }
    }
    return acc / (double)N - 1.0;
}

double vref_p2(int64_t N, int64_t a, int dim) {
    if (N < 1) return NAN;
    double* b = b2_table(N);
    if (!b) return NAN;
    const double v = p2_with_table(N, a, dim, b);
    free(b);
    return v;
}

int64_t vref_korobov_a(int64_t N) {
    if (N < 4) return 1;
    double* b = b2_table(N);
    if (!b) return -1;
    const int64_t amax = N / 2;
    double* crit = (double*)malloc(sizeof(double) * (size_t)(amax + 1));
    if (!crit) {
        free(b);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t a = 2; a <= amax; ++a) {
        crit[a] = (gcd64(a, N) == 1) ? p2_with_table(N, a, VREF_P2_DIM, b) : INFINITY;
    }
    int64_t best = -1;
    double best_v = INFINITY;
    for (int64_t a = 2; a <= amax; ++a) {
        if (crit[a] < best_v) {
            best_v = crit[a];
            best = a;
        }
    }
    free(crit);
    free(b);
    return best < 0 ? 1 : best;
}

int vref_lattice(int64_t N, int dim, uint32_t* g) {
    if (N < 1 || N > 0x7fffffff || dim < 0 || (dim > 0 && !g)) return VREF_ERR_ARG;
    const int64_t a = vref_korobov_a(N);
    if (a < 1) return VREF_ERR_ARG;
    int64_t gj = 1 % N;
    for (int j = 0; j < dim; ++j) {
        g[j] = (uint32_t)gj;
        gj = (gj * a) % N;
    }
    return VREF_OK;
}

/* ======================================================================== */
/* Covariance and Cholesky                                                   */
/* ======================================================================== */

double vref_cov(int kind, double variance, double range, double nu, double h) {
    if (kind == VREF_COV_EXPONENTIAL) return variance * exp(-h / range);
    if (kind == VREF_COV_MATERN) {
        if (nu == 0.5) return variance * exp(-h / range);
        if (nu == 1.5) {
            const double a = sqrt(3.0) * h / range;
            return variance * (1.0 + a) * exp(-a);
        }
        if (nu == 2.5) {
            const double a = sqrt(5.0) * h / range;
            return variance * (1.0 + a + a * a / 3.0) * exp(-a);
        }
    }
    return NAN;
}

int vref_cov_matrix(const double* sites, int64_t n, int kind, double variance, double range,
                    double nu, double nugget, double* Sigma) {
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t c = 0; c < n; ++c) {
            const double dx = sites[2 * a] - sites[2 * c];
            const double dy = sites[2 * a + 1] - sites[2 * c + 1];
            const double h = sqrt(dx * dx + dy * dy);
            double v = vref_cov(kind, variance, range, nu, h);
            if (a == c) v += nugget;
            if (isnan(v)) return VREF_ERR_ARG;
            Sigma[a * n + c] = v;
        }
    }
    return VREF_OK;
}

int vref_cholesky(int d, const double* A, double* L) {
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int t = 0; t < d; ++t) {
        for (int j = 0; j < t; ++j) {
            double s = A[t * d + j];
            for (int k = 0; k < j; ++k) s = fma(-L[t * d + k], L[j * d + k], s);
            L[t * d + j] = s / L[j * d + j];
        }
        double s = A[t * d + t];
        for (int k = 0; k < t; ++k) s = fma(-L[t * d + k], L[t * d + k], s);
        if (!(s > 0.0)) return VREF_ERR_NOT_PD;
        L[t * d + t] = sqrt(s);
    }
    return VREF_OK;
}

/* ======================================================================== */
/* Ordering and neighbours                                                   */
/* ======================================================================== */

int vref_quantize(const double* sites, int64_t D, int64_t* q) {
    if (D < 0 || (D > 0 && (!sites || !q))) return VREF_ERR_ARG;
    if (D == 0) return VREF_OK;
    double xmin = sites[0], xmax = sites[0], ymin = sites[1], ymax = sites[1];
    for (int64_t i = 1; i < D; ++i) {
        const double x = sites[2 * i], y = sites[2 * i + 1];
        if (x < xmin) xmin = x;
        if (x > xmax) xmax = x;
        if (y < ymin) ymin = y;
        if (y > ymax) ymax = y;
    }
    const double ex = xmax - xmin, ey = ymax - ymin;
    const double s = (ex > ey) ? ex : ey;
    if (!(s > 0.0)) {
        for (int64_t i = 0; i < 2 * D; ++i) q[i] = 0;
        return VREF_OK;
    }
    const double c = 1073741824.0 / s;
    for (int64_t i = 0; i < D; ++i) {
        const double tx = sites[2 * i] - xmin;
        const double ty = sites[2 * i + 1] - ymin;
        const double sx = tx * c;
        const double sy = ty * c;
        q[2 * i] = (int64_t)floor(sx);
        q[2 * i + 1] = (int64_t)floor(sy);
    }
    return VREF_OK;
}

static const double* g_sort_sites; /* comparator context (single-threaded use) */

static int cmp_xy(const void* pa, const void* pb) {
    const int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    const double xa = g_sort_sites[2 * a], xb = g_sort_sites[2 * b];
    if (xa < xb) return -1;
    if (xa > xb) return 1;
    const double ya = g_sort_sites[2 * a + 1], yb = g_sort_sites[2 * b + 1];
    if (ya < yb) return -1;
    if (ya > yb) return 1;
    return (a < b) ? -1 : (a > b);
}

static int64_t qd2(const int64_t* q, int64_t a, int64_t b) {
    const int64_t dx = q[2 * a] - q[2 * b];
    const int64_t dy = q[2 * a + 1] - q[2 * b + 1];
    return dx * dx + dy * dy;
}

int vref_order(const double* sites, int64_t D, int kind, int32_t* perm) {
    if (D < 0 || (D > 0 && (!sites || !perm)) || D > 0x7fffffff) return VREF_ERR_ARG;
    for (int64_t i = 0; i < D; ++i) perm[i] = (int32_t)i;
    if (kind == VREF_ORDER_IDENTITY || D == 0) return VREF_OK;
    if (kind == VREF_ORDER_XY) {
        g_sort_sites = sites;
        qsort(perm, (size_t)D, sizeof(int32_t), cmp_xy);
        return VREF_OK;
    }
    if (kind != VREF_ORDER_MAXMIN) return VREF_ERR_ARG;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)D);
    int64_t* mind = (int64_t*)malloc(sizeof(int64_t) * (size_t)D);
    char* chosen = (char*)calloc((size_t)D, 1);
    if (!q || !mind || !chosen) {
        free(q);
        free(mind);
        free(chosen);
        return VREF_ERR_ARG;
    }
    vref_quantize(sites, D, q);
    int64_t qxmax = 0, qymax = 0;
    for (int64_t i = 0; i < D; ++i) {
        if (q[2 * i] > qxmax) qxmax = q[2 * i];
        if (q[2 * i + 1] > qymax) qymax = q[2 * i + 1];
    }
    /* first: nearest to the box centre, compared as (2q - qmax)^2 sums */
    int64_t first = 0, best = -1;
    for (int64_t i = 0; i < D; ++i) {
        const int64_t dx = 2 * q[2 * i] - qxmax, dy = 2 * q[2 * i + 1] - qymax;
        const int64_t v = dx * dx + dy * dy;
        if (best < 0 || v < best) {
            best = v;
            first = i;
        }
    }
    perm[0] = (int32_t)first;
    chosen[first] = 1;
    for (int64_t i = 0; i < D; ++i) mind[i] = qd2(q, i, first);
    for (int64_t pos = 1; pos < D; ++pos) {
        int64_t pick = -1, pick_v = -1;
        for (int64_t i = 0; i < D; ++i) {
            if (chosen[i]) continue;
            if (mind[i] > pick_v) {
                pick_v = mind[i];
                pick = i;
            }
        }
        perm[pos] = (int32_t)pick;
        chosen[pick] = 1;
        for (int64_t i = 0; i < D; ++i) {
            if (chosen[i]) continue;
            const int64_t v = qd2(q, i, pick);
            if (v < mind[i]) mind[i] = v;
        }
    }
    free(q);
    free(mind);
    free(chosen);
    return VREF_OK;
}

static int cmp_i32(const void* pa, const void* pb) {
    const int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    return (a < b) ? -1 : (a > b);
}

/* The min(m, lim) smallest (d^2, j) keys of site i among j < lim, then listed
 * ascending in j (out has m entries, -1 padded). */
static void neighbors_lim(const int64_t* q, int64_t i, int64_t lim, int m, int32_t* out) {
    const int64_t cnt = (lim < m) ? lim : m;
    int64_t* kd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cnt + 1));
    int32_t* kj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt + 1));
    int64_t n = 0;
    for (int64_t j = 0; j < lim && cnt > 0; ++j) {
        const int64_t d2 = qd2(q, i, j);
        /* j ascending, so an equal d^2 never displaces an earlier entry */
        if (n == cnt && !(d2 < kd[n - 1])) continue;
        int64_t pos = (n < cnt) ? n : cnt - 1;
        if (n < cnt) ++n;
        while (pos > 0 && kd[pos - 1] > d2) {
            kd[pos] = kd[pos - 1];
            kj[pos] = kj[pos - 1];
            --pos;
        }
        kd[pos] = d2;
        kj[pos] = (int32_t)j;
    }
    qsort(kj, (size_t)n, sizeof(int32_t), cmp_i32);
    for (int r = 0; r < m; ++r) out[r] = (r < n) ? kj[r] : -1;
    free(kd);
    free(kj);
}

/* N_i: the min(m, i) nearest previously ordered sites (Sec. 2.1). */
static void neighbors_one(const int64_t* q, int64_t i, int m, int32_t* out) {
    neighbors_lim(q, i, i, m, out);
}

int vref_neighbors_of(const double* sites, int64_t D, int64_t i, int m, int32_t* out) {
    if (D < 1 || i < 0 || i >= D || m < 0 || !sites || (m > 0 && !out)) return VREF_ERR_ARG;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)D);
    if (!q) return VREF_ERR_ARG;
    vref_quantize(sites, D, q);
    neighbors_one(q, i, m, out);
    free(q);
    return VREF_OK;
}

int vref_neighbors(const double* sites, int64_t D, int m, int32_t* nbr) {
    if (D < 0 || m < 0 || (D > 0 && (!sites || (m > 0 && !nbr)))) return VREF_ERR_ARG;
    if (D == 0 || m == 0) return VREF_OK;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)D);
    if (!q) return VREF_ERR_ARG;
    vref_quantize(sites, D, q);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < D; ++i) neighbors_one(q, i, m, nbr + i * m);
    free(q);
    return VREF_OK;
}

/* ======================================================================== */
/* Genz separation-of-variables QMC                                          */
/* ======================================================================== */

typedef struct {
    double sum, comp;
} neumaier_t;

static void neumaier_add(neumaier_t* a, double x) {
    const double t = a->sum + x;
    if (fabs(a->sum) >= fabs(x))
        a->comp += (a->sum - t) + x;
    else
        a->comp += (x - t) + a->sum;
    a->sum = t;
}

/* e = Phi(z) and ec = 1 - Phi(z), the smaller of the two to full precision */
static void phi_pair(double z, double* e, double* ec) {
    const double t = vref_Phi_tail(z);
    if (z < 0.0) {
        *e = t;
        *ec = 1.0 - t;
    } else {
        *e = 1.0 - t;
        *ec = t;
    }
}

int vref_genz_sums(int d, const double* Sigma, const double* u, int64_t N, int S,
                   const uint32_t* g, const double* delta, int dim, double* num, double* den) {
    if (d < 1 || N < 1 || S < 1 || dim < d - 1 || !Sigma || !u || !num || !den) return VREF_ERR_ARG;
    if (d > 1 && (!g || !delta)) return VREF_ERR_ARG;
    double* L = (double*)malloc(sizeof(double) * (size_t)d * d);
    double* y = (double*)malloc(sizeof(double) * (size_t)(d > 1 ? d - 1 : 1));
    if (!L || !y) {
        free(L);
        free(y);
        return VREF_ERR_ARG;
    }
    const int st = vref_cholesky(d, Sigma, L);
    if (st != VREF_OK) {
        free(L);
        free(y);
        return st;
    }
    /* first conditional probability: no lattice coordinate (Eq. vecchia-cdf, Phi(x_1)) */
    double e0, ec0;
    phi_pair(u[0] / L[0], &e0, &ec0);
    if (d == 1) {
        for (int s = 0; s < S; ++s) {
            num[s] = e0;
            den[s] = 1.0;
        }
        free(L);
        free(y);
        return VREF_OK;
    }
    for (int s = 0; s < S; ++s) {
        neumaier_t acc_num = {0.0, 0.0}, acc_den = {0.0, 0.0};
        for (int64_t k = 0; k < N; ++k) {
            double e = e0, ec = ec0, f = 1.0;
            for (int t = 0; t + 1 < d; ++t) {
                f *= e; /* f = e_0 ... e_t */
                const uint64_t r = ((uint64_t)k * (uint64_t)g[t]) % (uint64_t)N;
                double x = (double)r / (double)N + delta[(int64_t)s * dim + t];
                if (x >= 1.0) x -= 1.0;
                const double a = fabs(2.0 * x - 1.0); /* tent transform: w = 1 - |2x - 1| */
                const double w = 1.0 - a;
                const double p = w * e;       /* w_t e_t */
                const double qq = a + w * ec; /* 1 - w_t e_t */
                y[t] = vref_Phiinv_pq(p, qq);
                double acc = u[t + 1];
                for (int j = 0; j <= t; ++j) acc = fma(-L[(t + 1) * d + j], y[j], acc);
                phi_pair(acc / L[(t + 1) * d + (t + 1)], &e, &ec);
            }
            neumaier_add(&acc_den, f);     /* e_0 ... e_{d-2}: the (d-1)-dim CDF sample */
            neumaier_add(&acc_num, f * e); /* times e_{d-1}: the d-dim CDF sample */
        }
        num[s] = (acc_num.sum + acc_num.comp) / (double)N;
        den[s] = (acc_den.sum + acc_den.comp) / (double)N;
    }
    free(L);
    free(y);
    return VREF_OK;
}

int vref_genz_cdf(int d, const double* Sigma, const double* u, int64_t N, int S, uint64_t seed,
                  double* p, double* rel_se) {
    if (d < 1 || S < 2 || N < 1 || !p || !rel_se) return VREF_ERR_ARG;
    const int dim = d > 1 ? d - 1 : 1;
    uint32_t* g = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)dim);
    double* delta = (double*)malloc(sizeof(double) * (size_t)S * dim);
    double* num = (double*)malloc(sizeof(double) * (size_t)S);
    double* den = (double*)malloc(sizeof(double) * (size_t)S);
    int st = (g && delta && num && den) ? VREF_OK : VREF_ERR_ARG;
    if (st == VREF_OK) st = vref_lattice(N, dim, g);
    if (st == VREF_OK) st = vref_shifts(seed, S, dim, delta);
    if (st == VREF_OK) st = vref_genz_sums(d, Sigma, u, N, S, g, delta, dim, num, den);
    if (st == VREF_OK) {
        double mean = 0.0;
        for (int s = 0; s < S; ++s) mean += num[s];
        mean /= (double)S;
        double ss = 0.0;
        for (int s = 0; s < S; ++s) ss += (num[s] - mean) * (num[s] - mean);
        *p = mean;
        *rel_se = sqrt(ss / ((double)S * (S - 1))) / mean;
    }
    free(g);
    free(delta);
    free(num);
    free(den);
    return st;
}

/* ======================================================================== */
/* The Vecchia log-CDF                                                       */
/* ======================================================================== */

int vref_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int check_cov(int kind, double variance, double range, double nu, double nugget) {
    if (!(variance > 0.0) || !(range > 0.0) || !(nugget >= 0.0)) return 0;
    if (kind == VREF_COV_EXPONENTIAL) return 1;
    if (kind == VREF_COV_MATERN) return nu == 0.5 || nu == 1.5 || nu == 2.5;
    return 0;
}

int vref_vecchia_partials(const double* sites, int64_t D, const int32_t* nbr, int m, int cov_kind,
                          double variance, double range, double nu, double nugget, const double* u,
                          int64_t N, int S, uint64_t seed, const int64_t* sites_idx, int64_t n_idx,
                          double* num, double* den, int64_t* bad_site) {
    if (D < 1 || m < 0 || N < 1 || S < 1 || !sites || !u || !num || !den) return VREF_ERR_ARG;
    if (m > 0 && !nbr) return VREF_ERR_ARG;
    if (!check_cov(cov_kind, variance, range, nu, nugget)) return VREF_ERR_ARG;
    const int64_t n = sites_idx ? n_idx : D;
    const int dim = m > 0 ? m : 1;
    uint32_t* g = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)dim);
    double* delta = (double*)malloc(sizeof(double) * (size_t)S * dim);
    if (!g || !delta) {
        free(g);
        free(delta);
        return VREF_ERR_ARG;
    }
    int st = vref_lattice(N, dim, g);
    if (st == VREF_OK) st = vref_shifts(seed, S, dim, delta);
    int64_t first_bad = -1;
    if (st == VREF_OK) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r = 0; r < n; ++r) {
            const int64_t i = sites_idx ? sites_idx[r] : r;
            if (i < 0 || i >= D) continue;
            const int q = (int)((i < m) ? i : m);
            const int d = q + 1;
            int64_t* b = (int64_t*)malloc(sizeof(int64_t) * (size_t)d);
            double* bs = (double*)malloc(sizeof(double) * 2 * (size_t)d);
            double* bu = (double*)malloc(sizeof(double) * (size_t)d);
            double* Sig = (double*)malloc(sizeof(double) * (size_t)d * d);
            int ok = b && bs && bu && Sig;
            /* block order (Sec. 2.2): N_i ascending, then i last, so that the
             * denominator's factor is the leading block of the numerator's */
            for (int a = 0; ok && a < q; ++a) {
                b[a] = nbr[i * m + a];
                if (b[a] < 0 || b[a] >= i || (a > 0 && b[a] <= b[a - 1])) ok = 0;
            }
            int lst = VREF_ERR_ARG;
            if (ok) {
                b[q] = i;
                for (int a = 0; a < d; ++a) {
                    bs[2 * a] = sites[2 * b[a]];
                    bs[2 * a + 1] = sites[2 * b[a] + 1];
                    bu[a] = u[b[a]];
                }
                lst = vref_cov_matrix(bs, d, cov_kind, variance, range, nu, nugget, Sig);
                if (lst == VREF_OK)
                    lst = vref_genz_sums(d, Sig, bu, N, S, g, delta, dim, num + r * S, den + r * S);
            }
            if (lst != VREF_OK) {
#pragma omp critical
                {
                    if (first_bad < 0 || i < first_bad) first_bad = i;
                    if (st == VREF_OK || lst == VREF_ERR_NOT_PD) st = lst;
                }
            }
            free(b);
            free(bs);
            free(bu);
            free(Sig);
        }
    }
    if (bad_site) *bad_site = first_bad;
    free(g);
    free(delta);
    return st;
}

int vref_vecchia_reduce(int64_t D, int S, const double* num, const double* den, double* log_p,
                        double* se, double* terms) {
    if (D < 1 || S < 2 || !num || !den || !log_p || !se) return VREF_ERR_ARG;
    double* nb = (double*)malloc(sizeof(double) * (size_t)D);
    double* db = (double*)malloc(sizeof(double) * (size_t)D);
    if (!nb || !db) {
        free(nb);
        free(db);
        return VREF_ERR_ARG;
    }
    double lp = 0.0;
    for (int64_t i = 0; i < D; ++i) {
        double sn = 0.0, sd = 0.0;
        for (int s = 0; s < S; ++s) {
            sn += num[i * S + s];
            sd += den[i * S + s];
        }
        nb[i] = sn / (double)S;
        db[i] = sd / (double)S;
        const double T = log(nb[i]) - log(db[i]); /* Sec. 3.1: each term on the log scale */
        if (terms) terms[i] = T;
        lp += T;
    }
    double ss = 0.0;
    for (int s = 0; s < S; ++s) {
        double l = 0.0;
        for (int64_t i = 0; i < D; ++i) l += num[i * S + s] / nb[i] - den[i * S + s] / db[i];
        ss += l * l;
    }
    *log_p = lp;
    *se = sqrt(ss / ((double)S * (double)(S - 1)));
    free(nb);
    free(db);
    return VREF_OK;
}

int vref_log_cdf(const double* sites, int64_t D, const int32_t* nbr, int m, int cov_kind,
                 double variance, double range, double nu, double nugget, const double* u,
                 int64_t N, int S, uint64_t seed, double* log_p, double* se, double* terms,
                 int64_t* bad_site) {
    if (D < 1 || S < 2) return VREF_ERR_ARG;
    double* num = (double*)malloc(sizeof(double) * (size_t)D * S);
    double* den = (double*)malloc(sizeof(double) * (size_t)D * S);
    if (!num || !den) {
        free(num);
        free(den);
        return VREF_ERR_ARG;
    }
    int st = vref_vecchia_partials(sites, D, nbr, m, cov_kind, variance, range, nu, nugget, u, N, S,
                                   seed, NULL, 0, num, den, bad_site);
    if (st == VREF_OK) st = vref_vecchia_reduce(D, S, num, den, log_p, se, terms);
    free(num);
    free(den);
    return st;
}

int vref_full_genz(const double* sites, int64_t D, int cov_kind, double variance, double range,
                   double nu, double nugget, const double* u, int64_t N, int S, uint64_t seed,
                   double* log_p, double* se) {
    if (D < 1 || S < 2 || !sites || !u || !log_p || !se) return VREF_ERR_ARG;
    if (!check_cov(cov_kind, variance, range, nu, nugget)) return VREF_ERR_ARG;
    double* Sig = (double*)malloc(sizeof(double) * (size_t)D * D);
    if (!Sig) return VREF_ERR_ARG;
    int st = vref_cov_matrix(sites, D, cov_kind, variance, range, nu, nugget, Sig);
    double p = 0.0, rse = 0.0;
    if (st == VREF_OK) st = vref_genz_cdf((int)D, Sig, u, N, S, seed, &p, &rse);
    if (st == VREF_OK) {
        *log_p = log(p);
        *se = rse;
    }
    free(Sig);
    return st;
}

/* ======================================================================== */
/* General terms: joint groups, general conditioning sets (Sec. 3.2)        */
/* ======================================================================== */

int vref_genz_sums_c(int d, int c, const double* Sigma, const double* u, int64_t N, int S,
                     const uint32_t* g, const double* delta, int dim, double* num, double* den) {
    if (d < 1 || c < 0 || c > d - 1 || N < 1 || S < 1 || dim < d - 1 || !Sigma || !u || !num || !den)
        return VREF_ERR_ARG;
    if (d > 1 && (!g || !delta)) return VREF_ERR_ARG;
    double* L = (double*)malloc(sizeof(double) * (size_t)d * d);
    double* y = (double*)malloc(sizeof(double) * (size_t)(d > 1 ? d - 1 : 1));
    if (!L || !y) {
        free(L);
        free(y);
        return VREF_ERR_ARG;
    }
    const int st = vref_cholesky(d, Sigma, L);
    if (st != VREF_OK) {
        free(L);
        free(y);
        return st;
    }
    double e0, ec0;
    phi_pair(u[0] / L[0], &e0, &ec0);
    for (int s = 0; s < S; ++s) {
        if (d == 1) { /* c = 0: the one-variable CDF, no lattice coordinate */
            num[s] = e0;
            den[s] = 1.0;
            continue;
        }
        neumaier_t acc_num = {0.0, 0.0}, acc_den = {0.0, 0.0};
        for (int64_t k = 0; k < N; ++k) {
            double e = e0, ec = ec0, f = 1.0, fc = 1.0;
            for (int t = 0; t + 1 < d; ++t) {
                f *= e; /* f = e_0 ... e_t */
                if (t + 1 == c) fc = f; /* the c-dim CDF sample of the leading block */
                const uint64_t r = ((uint64_t)k * (uint64_t)g[t]) % (uint64_t)N;
                double x = (double)r / (double)N + delta[(int64_t)s * dim + t];
                if (x >= 1.0) x -= 1.0;
                const double a = fabs(2.0 * x - 1.0);
                const double w = 1.0 - a;
                y[t] = vref_Phiinv_pq(w * e, a + w * ec);
                double acc = u[t + 1];
                for (int j = 0; j <= t; ++j) acc = fma(-L[(t + 1) * d + j], y[j], acc);
                phi_pair(acc / L[(t + 1) * d + (t + 1)], &e, &ec);
            }
            neumaier_add(&acc_num, f * e);
            if (c > 0) neumaier_add(&acc_den, fc);
        }
        num[s] = (acc_num.sum + acc_num.comp) / (double)N;
        den[s] = (c > 0) ? (acc_den.sum + acc_den.comp) / (double)N : 1.0;
    }
    free(L);
    free(y);
    return VREF_OK;
}

static int cmp_i32_asc(const void* pa, const void* pb) {
    const int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    return (a < b) ? -1 : (a > b);
}

/* sort ascending and drop repeats; returns the new length */
static int sort_unique(int32_t* v, int n) {
    qsort(v, (size_t)n, sizeof(int32_t), cmp_i32_asc);
    int w = 0;
    for (int r = 0; r < n; ++r)
        if (w == 0 || v[r] != v[w - 1]) v[w++] = v[r];
    return w;
}

int vref_group_cond_nearest(const double* sites, int64_t D, int p, int m, int cmax, int32_t* cond,
                            int32_t* count) {
    if (D < 1 || p < 1 || m < 0 || cmax < 0 || !sites || !count || (cmax > 0 && !cond))
        return VREF_ERR_ARG;
    const int64_t G = (D + p - 1) / p;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)D);
    if (!q) return VREF_ERR_ARG;
    vref_quantize(sites, D, q);
    int st = VREF_OK;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < G; ++k) {
        const int64_t i0 = k * p, i1 = (i0 + p < D) ? i0 + p : D;
        const int n_all = (int)(i1 - i0) * (m > 0 ? m : 1);
        int32_t* all = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_all);
        int32_t* one = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
        int n = 0;
        for (int64_t i = i0; i < i1 && m > 0; ++i) {
            neighbors_lim(q, i, i0, m, one); /* among the sites before the group */
            for (int r = 0; r < m; ++r)
                if (one[r] >= 0) all[n++] = one[r];
        }
        n = sort_unique(all, n);
        if (n > cmax) {
#pragma omp critical
            st = VREF_ERR_ARG;
        } else {
            for (int r = 0; r < cmax; ++r) cond[k * cmax + r] = (r < n) ? all[r] : -1;
            count[k] = n;
        }
        free(all);
        free(one);
    }
    free(q);
    return st;
}

int vref_group_cond_random(int64_t D, int p, int kk, uint64_t seed, int cmax, int32_t* cond,
                           int32_t* count) {
    if (D < 1 || D > 0x7fffffff || p < 1 || kk < 0 || kk > cmax || !count || (cmax > 0 && !cond))
        return VREF_ERR_ARG;
    const int64_t G = (D + p - 1) / p;
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    int32_t* set = (int32_t*)malloc(sizeof(int32_t) * (size_t)(kk > 0 ? kk : 1));
    if (!set) return VREF_ERR_ARG;
    for (int64_t k = 0; k < G; ++k) {
        const int64_t n = k * p; /* previously ordered sites */
        const int take = (int)((kk < n) ? kk : n);
        /* Floyd's sampling of `take` distinct indices from [0, n): for
         * j = n - take .. n - 1 draw t uniform in [0, j]; keep t unless it
         * is already in the set, else keep j. */
        int have = 0;
        for (int r = 0; r < take; ++r) {
            const int64_t j = n - take + r;
            const uint32_t ctr[4] = {(uint32_t)k, (uint32_t)r, 0x52C5u, (uint32_t)((uint64_t)k >> 32)};
            uint32_t o[4];
            vref_philox4x32_10(ctr, key, o);
            const int32_t t = (int32_t)(((uint64_t)o[0] * (uint64_t)(j + 1)) >> 32);
            int dup = 0;
            for (int a = 0; a < have; ++a)
                if (set[a] == t) dup = 1;
            set[have++] = dup ? (int32_t)j : t;
        }
        qsort(set, (size_t)have, sizeof(int32_t), cmp_i32_asc);
        for (int r = 0; r < cmax; ++r) cond[k * cmax + r] = (r < have) ? set[r] : -1;
        count[k] = have;
    }
    free(set);
    return VREF_OK;
}

double vref_aniso_h(double dx, double dy, double angle, double aspect) {
    /* Omega = (s_i - s_j)^T R(angle)^{-1} diag(1, aspect), h^2 = Omega Omega^T (Sec. 4.1) */
    const double c = cos(angle), s = sin(angle);
    const double o1 = dx * c - dy * s;
    const double o2 = aspect * (dx * s + dy * c);
    return sqrt(o1 * o1 + o2 * o2);
}

static int check_cov_t(const vref_cov_t* cv) {
    if (cv->kind == VREF_COV_ANISO_EXP)
        return cv->variance > 0.0 && cv->range > 0.0 && cv->nugget >= 0.0 && isfinite(cv->angle) &&
               cv->aspect > 0.0;
    return check_cov(cv->kind, cv->variance, cv->range, cv->nu, cv->nugget);
}

int vref_cov_matrix_t(const double* sites, int64_t n, const vref_cov_t* cv, double* Sigma) {
    if (!check_cov_t(cv)) return VREF_ERR_ARG;
    if (cv->kind != VREF_COV_ANISO_EXP)
        return vref_cov_matrix(sites, n, cv->kind, cv->variance, cv->range, cv->nu, cv->nugget, Sigma);
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t c = 0; c < n; ++c) {
            const double h = vref_aniso_h(sites[2 * a] - sites[2 * c], sites[2 * a + 1] - sites[2 * c + 1],
                                          cv->angle, cv->aspect);
            double v = cv->variance * exp(-h / cv->range);
            if (a == c) v += cv->nugget;
            Sigma[a * n + c] = v;
        }
    }
    return VREF_OK;
}

int vref_grouped_partials(const double* sites, int64_t D, int p, const int32_t* cond, int cmax,
                          const vref_cov_t* cv, const double* u, int64_t N, int S, uint64_t seed,
                          double* num, double* den, int64_t* bad_term) {
    if (D < 1 || p < 1 || cmax < 0 || N < 1 || S < 1 || !sites || !u || !num || !den || !cv)
        return VREF_ERR_ARG;
    if (cmax > 0 && !cond) return VREF_ERR_ARG;
    if (!check_cov_t(cv)) return VREF_ERR_ARG;
    const int64_t G = (D + p - 1) / p;
    const int dim = (cmax + p - 1 > 0) ? cmax + p - 1 : 1;
    uint32_t* g = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)dim);
    double* delta = (double*)malloc(sizeof(double) * (size_t)S * dim);
    if (!g || !delta) {
        free(g);
        free(delta);
        return VREF_ERR_ARG;
    }
    int st = vref_lattice(N, dim, g);
    if (st == VREF_OK) st = vref_shifts(seed, S, dim, delta);
    int64_t first_bad = -1;
    if (st == VREF_OK) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t k = 0; k < G; ++k) {
            const int64_t i0 = k * p, i1 = (i0 + p < D) ? i0 + p : D;
            int c = 0;
            while (c < cmax && cond[k * cmax + c] >= 0) ++c;
            const int d = c + (int)(i1 - i0);
            int64_t* b = (int64_t*)malloc(sizeof(int64_t) * (size_t)d);
            double* bs = (double*)malloc(sizeof(double) * 2 * (size_t)d);
            double* bu = (double*)malloc(sizeof(double) * (size_t)d);
            double* Sig = (double*)malloc(sizeof(double) * (size_t)d * d);
            int ok = b && bs && bu && Sig;
            /* block (C_k ascending, then the group's sites): the conditioning
             * CDF is the leading c-dim block of the joint one */
            for (int a = 0; ok && a < c; ++a) {
                b[a] = cond[k * cmax + a];
                if (b[a] >= i0 || (a > 0 && b[a] <= b[a - 1])) ok = 0;
            }
            for (int a = c; ok && a < cmax; ++a)
                if (cond[k * cmax + a] >= 0) ok = 0;
            int lst = VREF_ERR_ARG;
            if (ok) {
                for (int a = c; a < d; ++a) b[a] = i0 + (a - c);
                for (int a = 0; a < d; ++a) {
                    bs[2 * a] = sites[2 * b[a]];
                    bs[2 * a + 1] = sites[2 * b[a] + 1];
                    bu[a] = u[b[a]];
                }
                lst = vref_cov_matrix_t(bs, d, cv, Sig);
                if (lst == VREF_OK)
                    lst = vref_genz_sums_c(d, c, Sig, bu, N, S, g, delta, dim, num + k * S, den + k * S);
            }
            if (lst != VREF_OK) {
#pragma omp critical
                {
                    if (first_bad < 0 || k < first_bad) first_bad = k;
                    if (st == VREF_OK || lst == VREF_ERR_NOT_PD) st = lst;
                }
            }
            free(b);
            free(bs);
            free(bu);
            free(Sig);
        }
    }
    if (bad_term) *bad_term = first_bad;
    free(g);
    free(delta);
    return st;
}

int vref_grouped_log_cdf(const double* sites, int64_t D, int p, const int32_t* cond, int cmax,
                         const vref_cov_t* cv, const double* u, int64_t N, int S, uint64_t seed,
                         double* log_p, double* se, double* terms, int64_t* bad_term) {
    if (D < 1 || p < 1 || S < 2) return VREF_ERR_ARG;
    const int64_t G = (D + p - 1) / p;
    double* num = (double*)malloc(sizeof(double) * (size_t)G * S);
    double* den = (double*)malloc(sizeof(double) * (size_t)G * S);
    if (!num || !den) {
        free(num);
        free(den);
        return VREF_ERR_ARG;
    }
    int st = vref_grouped_partials(sites, D, p, cond, cmax, cv, u, N, S, seed, num, den, bad_term);
    if (st == VREF_OK) st = vref_vecchia_reduce(G, S, num, den, log_p, se, terms);
    free(num);
    free(den);
    return st;
}
