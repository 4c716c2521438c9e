"""The oracle: plain FP64 CPU restatement of the Vecchia Gaussian-CDF method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference legs may import this package.  It
shares no code with ``paper_2007_15195_gb300`` (the CUDA library); the two
meet only through the seeded inputs of ``paper_2007_15195_gb300.inputs``.

Each wrapper below calls the C routine of the same name in ``vref.c``; the
C header states which passage of the paper each routine follows.
"""
import ctypes as C
import os

import numpy as np

from .build import build as _build

_lib = None

OK, ERR_ARG, ERR_NOT_PD = 0, -1, -4
COV_EXPONENTIAL, COV_MATERN = 0, 1
ORDER_XY, ORDER_MAXMIN, ORDER_IDENTITY = 0, 1, 2

_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_u32p = C.POINTER(C.c_uint32)


COV_ANISO_EXP = 2


class CovT(C.Structure):
    """vref_cov_t: kind, variance, range, nu, nugget, angle, aspect."""
    _fields_ = [("kind", C.c_int), ("variance", C.c_double), ("range", C.c_double), ("nu", C.c_double),
                ("nugget", C.c_double), ("angle", C.c_double), ("aspect", C.c_double)]


def _cov_t(cov):
    """A covariance tuple (kind, variance, range, nu, nugget[, angle, aspect])."""
    c = tuple(cov) + (0.0, 1.0)[len(cov) - 5:] if len(cov) < 7 else tuple(cov)
    return CovT(int(c[0]), *[float(x) for x in c[1:7]])


class OracleError(RuntimeError):
    def __init__(self, status, where, site=-1):
        super().__init__("oracle %s returned %d%s" % (where, status,
                                                      "" if site < 0 else " (site %d)" % site))
        self.status = status
        self.site = site


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        L.vref_Phi.restype = C.c_double
        L.vref_Phi.argtypes = [C.c_double]
        L.vref_Phi_tail.restype = C.c_double
        L.vref_Phi_tail.argtypes = [C.c_double]
        L.vref_Phiinv.restype = C.c_double
        L.vref_Phiinv.argtypes = [C.c_double]
        L.vref_Phiinv_pq.restype = C.c_double
        L.vref_Phiinv_pq.argtypes = [C.c_double, C.c_double]
        L.vref_Phiinv_lower.restype = C.c_double
        L.vref_Phiinv_lower.argtypes = [C.c_double]
        L.vref_philox4x32_10.restype = None
        L.vref_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.vref_shifts.argtypes = [C.c_uint64, C.c_int, C.c_int, _dp]
        L.vref_p2.restype = C.c_double
        L.vref_p2.argtypes = [C.c_int64, C.c_int64, C.c_int]
        L.vref_korobov_a.restype = C.c_int64
        L.vref_korobov_a.argtypes = [C.c_int64]
        L.vref_lattice.argtypes = [C.c_int64, C.c_int, _u32p]
        L.vref_cov.restype = C.c_double
        L.vref_cov.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.vref_cov_matrix.argtypes = [_dp, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_double, _dp]
        L.vref_cholesky.argtypes = [C.c_int, _dp, _dp]
        L.vref_quantize.argtypes = [_dp, C.c_int64, _i64p]
        L.vref_order.argtypes = [_dp, C.c_int64, C.c_int, _i32p]
        L.vref_neighbors.argtypes = [_dp, C.c_int64, C.c_int, _i32p]
        L.vref_neighbors_of.argtypes = [_dp, C.c_int64, C.c_int64, C.c_int, _i32p]
        L.vref_genz_sums.argtypes = [C.c_int, _dp, _dp, C.c_int64, C.c_int, _u32p, _dp, C.c_int,
                                     _dp, _dp]
        L.vref_genz_cdf.argtypes = [C.c_int, _dp, _dp, C.c_int64, C.c_int, C.c_uint64, _dp, _dp]
        L.vref_vecchia_partials.argtypes = [_dp, C.c_int64, _i32p, C.c_int, C.c_int, C.c_double,
                                            C.c_double, C.c_double, C.c_double, _dp, C.c_int64,
                                            C.c_int, C.c_uint64, _i64p, C.c_int64, _dp, _dp, _i64p]
        L.vref_vecchia_reduce.argtypes = [C.c_int64, C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.vref_log_cdf.argtypes = [_dp, C.c_int64, _i32p, C.c_int, C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double, _dp, C.c_int64, C.c_int, C.c_uint64, _dp,
                                   _dp, _dp, _i64p]
        L.vref_full_genz.argtypes = [_dp, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_double, _dp, C.c_int64, C.c_int, C.c_uint64, _dp, _dp]
        L.vref_genz_sums_c.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_int64, C.c_int, _u32p, _dp,
                                       C.c_int, _dp, _dp]
        L.vref_group_cond_nearest.argtypes = [_dp, C.c_int64, C.c_int, C.c_int, C.c_int, _i32p, _i32p]
        L.vref_group_cond_random.argtypes = [C.c_int64, C.c_int, C.c_int, C.c_uint64, C.c_int, _i32p,
                                             _i32p]
        L.vref_aniso_h.restype = C.c_double
        L.vref_aniso_h.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.vref_cov_matrix_t.argtypes = [_dp, C.c_int64, C.POINTER(CovT), _dp]
        L.vref_grouped_partials.argtypes = [_dp, C.c_int64, C.c_int, _i32p, C.c_int, C.POINTER(CovT), _dp,
                                            C.c_int64, C.c_int, C.c_uint64, _dp, _dp, _i64p]
        L.vref_grouped_log_cdf.argtypes = [_dp, C.c_int64, C.c_int, _i32p, C.c_int, C.POINTER(CovT), _dp,
                                           C.c_int64, C.c_int, C.c_uint64, _dp, _dp, _dp, _i64p]
        L.vref_num_threads.restype = C.c_int
        L.vref_num_threads.argtypes = []
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _check(st, where, site=-1):
    if st != OK:
        raise OracleError(st, where, site)


# ---- univariate normal -------------------------------------------------------
def Phi(x):
    return lib().vref_Phi(float(x))


def Phi_tail(x):
    return lib().vref_Phi_tail(float(x))


def Phiinv(p):
    return lib().vref_Phiinv(float(p))


def Phiinv_pq(p, q):
    return lib().vref_Phiinv_pq(float(p), float(q))


# ---- Philox / shifts / lattice ----------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().vref_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def shifts(seed, S, dim):
    out = np.zeros((S, dim), dtype=np.float64)
    _check(lib().vref_shifts(C.c_uint64(seed), S, dim, _ptr(out, _dp)), "shifts")
    return out


def p2(N, a, dim=30):
    return lib().vref_p2(N, a, dim)


_korobov_cache = {}


def korobov_a(N):
    if N not in _korobov_cache:
        _korobov_cache[N] = lib().vref_korobov_a(N)
    return _korobov_cache[N]


def lattice(N, dim):
    a = korobov_a(N)
    g = np.zeros(dim, dtype=np.uint32)
    v = 1 % N
    for j in range(dim):
        g[j] = v
        v = (v * a) % N
    return g


def lattice_c(N, dim):
    """The C routine itself (recomputes the multiplier)."""
    g = np.zeros(dim, dtype=np.uint32)
    _check(lib().vref_lattice(N, dim, _ptr(g, _u32p)), "lattice")
    return g


# ---- covariance / Cholesky ---------------------------------------------------
def cov(kind, variance, range_, nu, h):
    return lib().vref_cov(kind, variance, range_, nu, float(h))


def cov_matrix(sites, kind, variance, range_, nu=0.5, nugget=0.0):
    s = _f64(sites).reshape(-1, 2)
    n = s.shape[0]
    out = np.zeros((n, n))
    _check(lib().vref_cov_matrix(_ptr(s, _dp), n, kind, variance, range_, nu, nugget,
                                 _ptr(out, _dp)), "cov_matrix")
    return out


def cholesky(A):
    A = _f64(A)
    d = A.shape[0]
    L = np.zeros_like(A)
    _check(lib().vref_cholesky(d, _ptr(A, _dp), _ptr(L, _dp)), "cholesky")
    return L


# ---- ordering / neighbours ---------------------------------------------------
def quantize(sites):
    s = _f64(sites).reshape(-1, 2)
    q = np.zeros(s.shape, dtype=np.int64)
    _check(lib().vref_quantize(_ptr(s, _dp), s.shape[0], _ptr(q, _i64p)), "quantize")
    return q


def order(sites, kind):
    s = _f64(sites).reshape(-1, 2)
    perm = np.zeros(s.shape[0], dtype=np.int32)
    _check(lib().vref_order(_ptr(s, _dp), s.shape[0], kind, _ptr(perm, _i32p)), "order")
    return perm


def neighbors(sites, m):
    s = _f64(sites).reshape(-1, 2)
    nbr = np.full((s.shape[0], max(m, 0)), -1, dtype=np.int32)
    _check(lib().vref_neighbors(_ptr(s, _dp), s.shape[0], m, _ptr(nbr, _i32p)), "neighbors")
    return nbr


def neighbors_of(sites, i, m):
    s = _f64(sites).reshape(-1, 2)
    out = np.full(max(m, 0), -1, dtype=np.int32)
    _check(lib().vref_neighbors_of(_ptr(s, _dp), s.shape[0], int(i), m, _ptr(out, _i32p)),
           "neighbors_of")
    return out


# ---- Genz --------------------------------------------------------------------
def genz_sums(Sigma, u, N, S, g, delta):
    Sig = _f64(Sigma)
    d = Sig.shape[0]
    u = _f64(u)
    g = np.ascontiguousarray(g, dtype=np.uint32)
    delta = _f64(delta)
    dim = delta.shape[1] if delta.ndim == 2 else 1
    num = np.zeros(S)
    den = np.zeros(S)
    _check(lib().vref_genz_sums(d, _ptr(Sig, _dp), _ptr(u, _dp), N, S, _ptr(g, _u32p),
                                _ptr(delta, _dp), dim, _ptr(num, _dp), _ptr(den, _dp)), "genz_sums")
    return num, den


def genz_cdf(Sigma, u, N, S, seed):
    Sig = _f64(Sigma)
    u = _f64(u)
    p = C.c_double()
    rse = C.c_double()
    _check(lib().vref_genz_cdf(Sig.shape[0], _ptr(Sig, _dp), _ptr(u, _dp), N, S, C.c_uint64(seed),
                               C.byref(p), C.byref(rse)), "genz_cdf")
    return p.value, rse.value


# ---- Vecchia -----------------------------------------------------------------
def _cov_args(cov):
    kind, variance, range_, nu, nugget = cov
    return int(kind), float(variance), float(range_), float(nu), float(nugget)


def vecchia_partials(sites, nbr, m, cov, u, N, S, seed, idx=None):
    s = _f64(sites).reshape(-1, 2)
    D = s.shape[0]
    nb = np.ascontiguousarray(nbr, dtype=np.int32) if m > 0 else np.zeros(1, np.int32)
    u = _f64(u)
    ix = None if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    n = D if ix is None else ix.shape[0]
    num = np.zeros((n, S))
    den = np.zeros((n, S))
    bad = C.c_int64(-1)
    st = lib().vref_vecchia_partials(_ptr(s, _dp), D, _ptr(nb, _i32p), m, *_cov_args(cov),
                                     _ptr(u, _dp), N, S, C.c_uint64(seed), _ptr(ix, _i64p),
                                     0 if ix is None else n, _ptr(num, _dp), _ptr(den, _dp),
                                     C.byref(bad))
    _check(st, "vecchia_partials", bad.value)
    return num, den


def vecchia_reduce(num, den):
    num = _f64(num)
    den = _f64(den)
    D, S = num.shape
    lp = C.c_double()
    se = C.c_double()
    terms = np.zeros(D)
    _check(lib().vref_vecchia_reduce(D, S, _ptr(num, _dp), _ptr(den, _dp), C.byref(lp),
                                     C.byref(se), _ptr(terms, _dp)), "vecchia_reduce")
    return lp.value, se.value, terms


def log_cdf(sites, nbr, m, cov, u, N, S, seed, return_terms=False):
    s = _f64(sites).reshape(-1, 2)
    D = s.shape[0]
    nb = np.ascontiguousarray(nbr, dtype=np.int32) if m > 0 else np.zeros(1, np.int32)
    u = _f64(u)
    lp = C.c_double()
    se = C.c_double()
    terms = np.zeros(D)
    bad = C.c_int64(-1)
    st = lib().vref_log_cdf(_ptr(s, _dp), D, _ptr(nb, _i32p), m, *_cov_args(cov), _ptr(u, _dp), N,
                            S, C.c_uint64(seed), C.byref(lp), C.byref(se), _ptr(terms, _dp),
                            C.byref(bad))
    _check(st, "log_cdf", bad.value)
    if return_terms:
        return lp.value, se.value, terms
    return lp.value, se.value


def full_genz(sites, cov, u, N, S, seed):
    s = _f64(sites).reshape(-1, 2)
    u = _f64(u)
    lp = C.c_double()
    se = C.c_double()
    _check(lib().vref_full_genz(_ptr(s, _dp), s.shape[0], *_cov_args(cov), _ptr(u, _dp), N, S,
                                C.c_uint64(seed), C.byref(lp), C.byref(se)), "full_genz")
    return lp.value, se.value


# ---- general terms: joint groups, conditioning sets (Sec. 3.2) ---------------
def genz_sums_c(Sigma, u, c, N, S, g, delta):
    Sig = _f64(Sigma)
    d = Sig.shape[0]
    u = _f64(u)
    g = np.ascontiguousarray(g, dtype=np.uint32)
    delta = _f64(delta)
    dim = delta.shape[1] if delta.ndim == 2 else 1
    num = np.zeros(S)
    den = np.zeros(S)
    _check(lib().vref_genz_sums_c(d, c, _ptr(Sig, _dp), _ptr(u, _dp), N, S, _ptr(g, _u32p),
                                  _ptr(delta, _dp), dim, _ptr(num, _dp), _ptr(den, _dp)), "genz_sums_c")
    return num, den


def group_cond_nearest(sites, p, m, cmax):
    s = _f64(sites).reshape(-1, 2)
    D = s.shape[0]
    G = (D + p - 1) // p
    cond = np.full((G, max(cmax, 1)), -1, dtype=np.int32)
    cnt = np.zeros(G, dtype=np.int32)
    _check(lib().vref_group_cond_nearest(_ptr(s, _dp), D, p, m, cmax, _ptr(cond, _i32p), _ptr(cnt, _i32p)),
           "group_cond_nearest")
    return cond[:, :cmax], cnt


def group_cond_random(D, p, kk, seed, cmax):
    G = (D + p - 1) // p
    cond = np.full((G, max(cmax, 1)), -1, dtype=np.int32)
    cnt = np.zeros(G, dtype=np.int32)
    _check(lib().vref_group_cond_random(D, p, kk, C.c_uint64(seed), cmax, _ptr(cond, _i32p),
                                        _ptr(cnt, _i32p)), "group_cond_random")
    return cond[:, :cmax], cnt


def aniso_h(dx, dy, angle, aspect):
    return lib().vref_aniso_h(float(dx), float(dy), float(angle), float(aspect))


def cov_matrix_t(sites, cov):
    s = _f64(sites).reshape(-1, 2)
    n = s.shape[0]
    out = np.zeros((n, n))
    cv = _cov_t(cov)
    _check(lib().vref_cov_matrix_t(_ptr(s, _dp), n, C.byref(cv), _ptr(out, _dp)), "cov_matrix_t")
    return out


def grouped_partials(sites, p, cond, cov, u, N, S, seed):
    s = _f64(sites).reshape(-1, 2)
    D = s.shape[0]
    G = (D + p - 1) // p
    cd = np.ascontiguousarray(cond, dtype=np.int32).reshape(G, -1)
    cmax = cd.shape[1]
    num = np.zeros((G, S))
    den = np.zeros((G, S))
    bad = C.c_int64(-1)
    cv = _cov_t(cov)
    st = lib().vref_grouped_partials(_ptr(s, _dp), D, p, _ptr(cd, _i32p) if cmax else None, cmax,
                                     C.byref(cv), _ptr(_f64(u), _dp), N, S, C.c_uint64(seed),
                                     _ptr(num, _dp), _ptr(den, _dp), C.byref(bad))
    _check(st, "grouped_partials", bad.value)
    return num, den


def grouped_log_cdf(sites, p, cond, cov, u, N, S, seed, return_terms=False):
    """log P ~ sum_k [log Phi(u_{C_k, G_k}) - log Phi(u_{C_k})] over the groups
    G_k of p consecutive ordered sites and their conditioning sets C_k (rows
    of cond, ascending, -1 padded)."""
    s = _f64(sites).reshape(-1, 2)
    D = s.shape[0]
    G = (D + p - 1) // p
    cd = np.ascontiguousarray(cond, dtype=np.int32).reshape(G, -1)
    cmax = cd.shape[1]
    lp = C.c_double()
    se = C.c_double()
    terms = np.zeros(G)
    bad = C.c_int64(-1)
    cv = _cov_t(cov)
    st = lib().vref_grouped_log_cdf(_ptr(s, _dp), D, p, _ptr(cd, _i32p) if cmax else None, cmax,
                                    C.byref(cv), _ptr(_f64(u), _dp), N, S, C.c_uint64(seed), C.byref(lp),
                                    C.byref(se), _ptr(terms, _dp), C.byref(bad))
    _check(st, "grouped_log_cdf", bad.value)
    if return_terms:
        return lp.value, se.value, terms
    return lp.value, se.value


def num_threads():
    return lib().vref_num_threads()


def set_threads(n):
    """Threads for later calls (OpenMP reads the variable at first parallel region)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))


# ---- scale mixture (Sec. 4, Eq. model01-model03) ----------------------------
def mixing_quantile(v, beta, gamma):
    """r = F_R^{-1}(v) for F_R(r) = 1 - exp(-gamma (r^beta - 1)/beta), r >= 1
    (Eq. model02, beta > 0) and its beta -> 0 limit 1 - r^(-gamma) (the
    printed "1 - r^gamma" read with the exponent's sign restored)."""
    L = -np.log1p(-np.asarray(v, dtype=np.float64))
    if beta > 0:
        return (1.0 + beta * L / gamma) ** (1.0 / beta)
    return np.exp(L / gamma)


def mixture_nodes(n_nodes):
    """Nodes v_q in (0, 1) and weights of the rule for int_0^1 f(v) dv: the
    substitution v = 1 - (1 - t)^4 (dv = 4 (1 - t)^3 dt), then Gauss-Legendre
    in t on [0, 1].  The substitution flattens the singularity of F_R^{-1} at
    v = 1."""
    t, w = np.polynomial.legendre.leggauss(n_nodes)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w * 4.0 * (1.0 - t) ** 3
    return 1.0 - (1.0 - t) ** 4, w


def mixture_log_cdf(sites, nbr, m, cov, x, N, S, seed, beta, gamma, n_nodes):
    """log G(x), G(x) = int Phi_D(x / r; Sigma) dF_R(r) (Eq. model03) =
    int_0^1 Phi_D(x / F_R^{-1}(v); Sigma) dv by the rule of mixture_nodes,
    each node's Vecchia log-CDF with the covariance scaled by r^2
    (Phi_D(x/r; Sigma) = Phi_D(x; r^2 Sigma)); written with numpy on top of
    log_cdf."""
    v, w = mixture_nodes(n_nodes)
    kind, var, rng_, nu, nug = cov
    terms = []
    for vq, wq in zip(v, w):
        r = float(mixing_quantile(vq, beta, gamma))
        lp, _ = log_cdf(sites, nbr, m, (kind, var * r * r, rng_, nu, nug * r * r), x, N, S, seed)
        terms.append(np.log(wq) + lp)
    terms = np.array(terms)
    mx = terms.max()
    return float(mx + np.log(np.sum(np.exp(terms - mx))))


# ---- censored likelihood G_I (Sec. 4, Eq. model05) ---------------------------
def vecchia_from_matrix(Sigma, nbr, m, u, N, S, seed, return_terms=False):
    """Eq. (vecchia-cdf) for N(0, Sigma) with Sigma given as a matrix: term i
    is the block (N_i ascending, i) of Sigma, by genz_sums on the lattice and
    shifts of dimension max(m, 1); reduced as vecchia_reduce."""
    Sigma = _f64(Sigma)
    u = _f64(u)
    D = Sigma.shape[0]
    dim = max(m, 1)
    g, dl = lattice(N, dim), shifts(seed, S, dim)
    num = np.zeros((D, S))
    den = np.zeros((D, S))
    for i in range(D):
        q = min(m, i)
        b = [int(j) for j in nbr[i, :q]] + [i]
        num[i], den[i] = genz_sums(Sigma[np.ix_(b, b)], u[b], N, S, g, dl)
    lp, se, terms = vecchia_reduce(num, den)
    return (lp, se, terms) if return_terms else (lp, se)


def censored_log_cdf(sites_c, nbr, m, sites_i, cov, x_c, x_i, N, S, seed, beta=0.5, gamma=1.0, n_nodes=16):
    """log G_I(x) of Eq. (model05): the observations x_I above the threshold
    enter through their density, the censored ones x_c through the CDF of
    their conditional law given x_I:
        G_I = int Phi_c{(x_c - mu)/r; Sigma_{c|I}} phi_k(x_I/r; Sigma_II) r^-k dF_R(r),
        mu = Sigma_cI Sigma_II^-1 x_I,  Sigma_{c|I} = Sigma_cc - Sigma_cI Sigma_II^-1 Sigma_Ic,
    with Phi_c by Eq. (vecchia-cdf) on the censored sites (ordered; rows nbr),
    Phi_c(y/r; A) = Phi_c(y; r^2 A), phi_k in closed form, and the integral by
    the rule of mixture_nodes; n_nodes = 0 means R = 1 (the Gaussian case).
    Linear algebra by numpy's LAPACK solves."""
    sc = _f64(sites_c).reshape(-1, 2)
    si = _f64(sites_i).reshape(-1, 2)
    xc, xi = _f64(x_c), _f64(x_i)
    c, k = sc.shape[0], si.shape[0]
    Sig = cov_matrix_t(np.concatenate([si, sc]), cov)
    Sii, Sic, Scc = Sig[:k, :k], Sig[:k, k:], Sig[k:, k:]
    if k:
        Scond = Scc - Sic.T @ np.linalg.solve(Sii, Sic)
        sol = np.linalg.solve(Sii, xi)
        mu = Sic.T @ sol
        quad = float(xi @ sol)
        logdet = float(np.linalg.slogdet(Sii)[1])
    else:
        Scond, mu, quad, logdet = Scc, np.zeros(c), 0.0, 0.0

    def node(r):
        lp = 0.0
        if c:
            lp, _ = vecchia_from_matrix(r * r * Scond, nbr, m, xc - mu, N, S, seed)
        # log phi_k(x_I / r; Sigma_II) - k log r
        ld = -0.5 * k * np.log(2 * np.pi) - 0.5 * logdet - quad / (2 * r * r) - k * np.log(r)
        return lp + ld

    if n_nodes == 0:
        return float(node(1.0))
    v, w = mixture_nodes(n_nodes)
    terms = np.array([np.log(wq) + node(float(mixing_quantile(vq, beta, gamma))) for vq, wq in zip(v, w)])
    mx = terms.max()
    return float(mx + np.log(np.sum(np.exp(terms - mx))))
