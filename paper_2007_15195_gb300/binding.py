"""ctypes binding of libvecchia: argument marshalling only.

Every function below has the name of the C entry point it calls
(include/vecchia.h) and does nothing but convert arrays to pointers and
status codes to exceptions; every step of the method runs in the library.
Arrays may be torch tensors (CPU or CUDA) or numpy arrays; outputs come back
on the same kind of container and device as the first array argument.
The library must have been built (``__graft_entry__.build()``); there is no
fallback implementation.
"""
import ctypes as C
import os

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the stack
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvecchia.so")

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_NOT_PD, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7)
ORDER_XY, ORDER_MAXMIN, ORDER_IDENTITY = 0, 1, 2
COV_EXPONENTIAL, COV_MATERN, COV_ANISO_EXP = 0, 1, 2
FP64, MIXED = 0, 1
COND_NEAREST, COND_RANDOM = 0, 1
MAX_M, MAX_S = 63, 64
ORDER_KINDS = {"xy": ORDER_XY, "maxmin": ORDER_MAXMIN, "identity": ORDER_IDENTITY}


class VecchiaError(RuntimeError):
    def __init__(self, status, where, site=-1):
        msg = "%s: %s (status %d)" % (where, strerror(status) if _lib else "error", status)
        if site >= 0:
            msg += ", ordered site %d" % site
        super().__init__(msg)
        self.status = status
        self.site = site


class vecchia_cov(C.Structure):
    _fields_ = [("kind", C.c_int32), ("variance", C.c_double), ("range", C.c_double),
                ("nu", C.c_double), ("nugget", C.c_double), ("angle", C.c_double), ("aspect", C.c_double)]


class vecchia_problem(C.Structure):
    _fields_ = [("sites", C.c_void_p), ("nbr", C.c_void_p), ("u", C.c_void_p), ("D", C.c_int64),
                ("m", C.c_int32), ("S", C.c_int32), ("N", C.c_int64), ("seed", C.c_uint64),
                ("cov", vecchia_cov), ("group", C.c_int32), ("cond_max", C.c_int32)]


class vecchia_segment(C.Structure):
    _fields_ = [("prob", vecchia_problem), ("num", C.c_void_p), ("den", C.c_void_p),
                ("result", C.c_void_p), ("site_begin", C.c_int64), ("site_count", C.c_int64)]


# host view of a vecchia_result slot (32 bytes)
RESULT_DTYPE = np.dtype([("log_p", "<f8"), ("std_err", "<f8"), ("bad_site", "<i8"), ("status", "<i4"),
                         ("reserved", "<i4")])

_lib = None
_vp = C.c_void_p


def lib():
    """Load libvecchia.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libvecchia is not built (%s missing); run __graft_entry__.build()"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        L.vecchia_strerror.restype = C.c_char_p
        L.vecchia_strerror.argtypes = [C.c_int]
        L.vecchia_create.argtypes = [C.POINTER(_vp), C.c_int, _vp]
        L.vecchia_destroy.argtypes = [_vp]
        L.vecchia_set_stream.argtypes = [_vp, _vp]
        L.vecchia_order.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp]
        L.vecchia_neighbors.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp]
        L.vecchia_apply_order.argtypes = [_vp, _vp, _vp, _vp, C.c_int64, _vp, _vp]
        L.vecchia_log_cdf.argtypes = [_vp, _vp, C.c_int64, _vp, C.c_int, vecchia_cov, _vp, C.c_int64,
                                      C.c_int, C.c_uint64, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]
        L.vecchia_log_cdf_terms.argtypes = [_vp, _vp, C.c_int64, _vp, C.c_int, vecchia_cov, _vp,
                                            C.c_int64, C.c_int, C.c_uint64, C.c_int,
                                            C.POINTER(C.c_double), C.POINTER(C.c_double), _vp, _vp,
                                            _vp]
        L.vecchia_log_cdf_batch.argtypes = [_vp, C.POINTER(vecchia_problem), C.c_int, C.c_int, _vp,
                                            _vp, _vp]
        L.vecchia_neighbors_async.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp]
        L.vecchia_result_init.argtypes = [_vp, _vp, C.c_int]
        L.vecchia_partials_async.argtypes = [_vp, C.POINTER(vecchia_segment), C.c_int, C.c_int]
        L.vecchia_reduce_async.argtypes = [_vp, C.POINTER(vecchia_segment), C.c_int]
        L.vecchia_plan_create.argtypes = [_vp, C.POINTER(vecchia_problem), C.c_int, C.c_int,
                                          C.POINTER(_vp), _vp]
        L.vecchia_plan_run.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.vecchia_plan_destroy.argtypes = [_vp]
        L.vecchia_mixture_log_cdf.argtypes = [_vp, _vp, C.c_int64, _vp, C.c_int, vecchia_cov, _vp,
                                              C.c_int64, C.c_int, C.c_uint64, C.c_double, C.c_double,
                                              C.c_int, C.c_int, C.POINTER(C.c_double),
                                              C.POINTER(C.c_double)]
        L.vecchia_group_conditioning.argtypes = [_vp, _vp, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                                 C.c_int, _vp, _vp]
        L.vecchia_grouped_log_cdf.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp, C.c_int, vecchia_cov, _vp,
                                              C.c_int64, C.c_int, C.c_uint64, C.c_int, C.POINTER(C.c_double),
                                              C.POINTER(C.c_double)]
        L.vecchia_full_genz.argtypes = [_vp, _vp, C.c_int64, vecchia_cov, _vp, C.c_int64, C.c_int, C.c_uint64,
                                        C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.vecchia_full_cholesky.argtypes = [_vp, _vp, C.c_int64, vecchia_cov, C.c_int, _vp]
        L.vecchia_censored_log_cdf.argtypes = [_vp, _vp, C.c_int64, _vp, C.c_int, _vp, C.c_int64, vecchia_cov, _vp,
                                               _vp, C.c_int64, C.c_int, C.c_uint64, C.c_double, C.c_double,
                                               C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.vecchia_log_cdf_unordered.argtypes = [_vp, _vp, _vp, C.c_int64, C.c_int, C.c_int, vecchia_cov, C.c_int64,
                                                C.c_int, C.c_uint64, C.c_int, _vp, C.POINTER(C.c_double),
                                                C.POINTER(C.c_double)]
        L.vecchia_lattice.argtypes = [C.c_int64, C.c_int, _vp]
        L.vecchia_shifts.argtypes = [C.c_uint64, C.c_int, C.c_int, _vp]
        L.vecchia_last_error_site.restype = C.c_int64
        L.vecchia_last_error_site.argtypes = [_vp]
        L.vecchia_set_tile.argtypes = [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.vecchia_reset_tiles.argtypes = [_vp]
        L.vecchia_set_timing.argtypes = [_vp, C.c_int]
        L.vecchia_eval_special.argtypes = [_vp, C.c_int, _vp, C.c_int64, _vp]
        L.vecchia_eval_special64.argtypes = [_vp, C.c_int, _vp, C.c_int64, _vp]
        L.vecchia_log_cdf_noalloc.argtypes = [C.c_int, _vp, _vp, C.c_int64, _vp, C.c_int, vecchia_cov,
                                              _vp, C.c_int64, C.c_int, C.c_uint64, C.c_int,
                                              C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.vecchia_genz_time_ms.argtypes = [_vp, C.POINTER(C.c_double)]
        L.vecchia_set_full_genz_wait.argtypes = [_vp, C.c_uint64, C.c_int]
        _lib = L
    return _lib


def strerror(status):
    return lib().vecchia_strerror(int(status)).decode()


# ------------------------------ marshalling ---------------------------------

def _is_torch(a):
    return torch is not None and isinstance(a, torch.Tensor)


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _as(a, np_dtype, torch_dtype):
    """Keep the container (torch on its device, else numpy); enforce dtype and contiguity."""
    if _is_torch(a):
        if a.dtype != torch_dtype:
            a = a.to(torch_dtype)
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np_dtype)


def _empty_like_kind(ref, shape, np_dtype, torch_dtype):
    if _is_torch(ref):
        return torch.empty(shape, dtype=torch_dtype, device=ref.device)
    return np.empty(shape, dtype=np_dtype)


def _f64(a):
    return _as(a, np.float64, torch.float64 if torch is not None else None)


def _i32(a):
    return _as(a, np.int32, torch.int32 if torch is not None else None)


def _check(st, where, ctx=None):
    if st != OK:
        site = lib().vecchia_last_error_site(ctx.handle) if ctx is not None and ctx.handle else -1
        raise VecchiaError(st, where, site)


def make_cov(kind=COV_EXPONENTIAL, variance=1.0, range_=0.1, nu=0.5, nugget=0.0, angle=0.0, aspect=1.0):
    """A vecchia_cov from arguments or a tuple (kind, variance, range, nu, nugget[, angle, aspect])."""
    if isinstance(kind, vecchia_cov):
        return kind
    if isinstance(kind, (tuple, list)):
        t = tuple(kind) + (0.0, 1.0)[len(kind) - 5:] if len(kind) < 7 else tuple(kind)
        kind, variance, range_, nu, nugget, angle, aspect = t
    return vecchia_cov(int(kind), float(variance), float(range_), float(nu), float(nugget), float(angle),
                       float(aspect))


# ------------------------------ the context ---------------------------------

class Context:
    """A libvecchia context bound to one CUDA device and stream."""

    def __init__(self, device=0, stream=None):
        self.device = int(device)
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream(self.device).cuda_stream
        h = _vp()
        _check(lib().vecchia_create(C.byref(h), self.device, _vp(stream or 0)), "vecchia_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().vecchia_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        _check(lib().vecchia_set_stream(self.handle, _vp(stream or 0)), "vecchia_set_stream", self)


def vecchia_create(device=0, stream=None):
    return Context(device, stream)


def vecchia_destroy(ctx):
    ctx.close()


def vecchia_order(ctx, sites, kind="maxmin"):
    s = _f64(sites)
    D = s.shape[0]
    k = ORDER_KINDS.get(kind, kind) if isinstance(kind, str) else int(kind)
    perm = _empty_like_kind(s, (D,), np.int32, torch.int32 if torch is not None else None)
    h = ctx.handle if ctx is not None else None
    _check(lib().vecchia_order(h, _ptr(s), D, k, _ptr(perm)), "vecchia_order", ctx)
    return perm


def vecchia_apply_order(ctx, perm, sites, u=None):
    """Returns (sites[perm], u[perm]) on the inputs' device (u may be None)."""
    s = _f64(sites)
    p = _i32(perm)
    D = s.shape[0]
    tdt = torch.float64 if torch is not None else None
    so = _empty_like_kind(s, (D, 2), np.float64, tdt)
    uu = _f64(u) if u is not None else None
    uo = _empty_like_kind(s, (D,), np.float64, tdt) if u is not None else None
    h = ctx.handle if ctx is not None else None
    _check(lib().vecchia_apply_order(h, _ptr(p), _ptr(s), _ptr(uu), D, _ptr(so), _ptr(uo)),
           "vecchia_apply_order", ctx)
    return so, uo


def vecchia_neighbors(ctx, sites_ordered, m):
    s = _f64(sites_ordered)
    D = s.shape[0]
    nbr = _empty_like_kind(s, (D, max(int(m), 0)), np.int32, torch.int32 if torch is not None else None)
    _check(lib().vecchia_neighbors(ctx.handle, _ptr(s), D, int(m), _ptr(nbr) if m > 0 else None),
           "vecchia_neighbors", ctx)
    return nbr


def vecchia_log_cdf(ctx, sites_ordered, nbr, m, cov, u, N, S, seed=0, precision=MIXED):
    s, uu = _f64(sites_ordered), _f64(u)
    nb = _i32(nbr) if m > 0 else None
    lp, se = C.c_double(), C.c_double()
    _check(lib().vecchia_log_cdf(ctx.handle, _ptr(s), s.shape[0], _ptr(nb), int(m), make_cov(cov),
                                 _ptr(uu), int(N), int(S), C.c_uint64(int(seed)), int(precision),
                                 C.byref(lp), C.byref(se)), "vecchia_log_cdf", ctx)
    return lp.value, se.value


def vecchia_group_conditioning(ctx, sites_ordered, p, m, method=COND_NEAREST, seed=0, cmax=None):
    """Conditioning rows of the groups of p consecutive ordered sites: returns
    (cond [ceil(D/p), cmax], count [ceil(D/p)]) on the sites' device (method
    COND_NEAREST: union of each member's m nearest earlier sites, cmax default
    p m; COND_RANDOM: m uniform earlier sites, cmax default m)."""
    s = _f64(sites_ordered)
    D = s.shape[0]
    p, m = int(p), int(m)
    if cmax is None:
        cmax = p * m if method == COND_NEAREST else m
    G = (D + p - 1) // p
    i32 = torch.int32 if torch is not None else None
    cond = _empty_like_kind(s, (G, max(int(cmax), 1)), np.int32, i32)
    cnt = _empty_like_kind(s, (G,), np.int32, i32)
    _check(lib().vecchia_group_conditioning(ctx.handle, _ptr(s), D, p, m, int(method), C.c_uint64(int(seed)),
                                            int(cmax), _ptr(cond), _ptr(cnt)), "vecchia_group_conditioning",
           ctx)
    return cond[:, :int(cmax)], cnt


def vecchia_grouped_log_cdf(ctx, sites_ordered, p, cond, cov, u, N, S, seed=0, precision=MIXED):
    """The joint-group Vecchia log-CDF (groups of p ordered sites, conditioning
    rows cond [ceil(D/p), cmax]); returns (log_p, std_err)."""
    s, uu = _f64(sites_ordered), _f64(u)
    cmax = int(cond.shape[1])
    cd = _i32(cond) if cmax > 0 else None
    lp, se = C.c_double(), C.c_double()
    _check(lib().vecchia_grouped_log_cdf(ctx.handle, _ptr(s), s.shape[0], int(p), _ptr(cd), cmax,
                                         make_cov(cov), _ptr(uu), int(N), int(S), C.c_uint64(int(seed)),
                                         int(precision), C.byref(lp), C.byref(se)), "vecchia_grouped_log_cdf",
           ctx)
    return lp.value, se.value


def vecchia_full_genz(ctx, sites_ordered, cov, u, N, S, seed=0, precision=MIXED):
    """The full D-dimensional Genz estimate: returns (log_p, rel_se)."""
    s, uu = _f64(sites_ordered), _f64(u)
    lp, se = C.c_double(), C.c_double()
    _check(lib().vecchia_full_genz(ctx.handle, _ptr(s), s.shape[0], make_cov(cov), _ptr(uu), int(N), int(S),
                                   C.c_uint64(int(seed)), int(precision), C.byref(lp), C.byref(se)),
           "vecchia_full_genz", ctx)
    return lp.value, se.value


def vecchia_full_cholesky(ctx, sites_ordered, cov, precision=MIXED, out=None):
    """Covariance factor behind vecchia_full_genz (diagnostic): returns the D x D
    array (lower triangle the factor, upper zeros), numpy unless `out` (a CUDA
    float64 tensor of D x D) is given."""
    s = _f64(sites_ordered)
    D = int(s.shape[0])
    L = out if out is not None else np.empty((D, D), dtype=np.float64)
    _check(lib().vecchia_full_cholesky(ctx.handle, _ptr(s), D, make_cov(cov), int(precision), _ptr(L)),
           "vecchia_full_cholesky", ctx)
    return L


def vecchia_censored_log_cdf(ctx, sites_c, nbr, m, sites_i, cov, x_c, x_i, N, S, seed=0, beta=0.5, gamma=1.0,
                             n_nodes=16, precision=MIXED):
    """Censored likelihood log G_I (censored sites_c/x_c with neighbour rows nbr,
    observed sites_i/x_i); n_nodes = 0 for R = 1.  Returns (log_g, std_err)."""
    sc, xc = _f64(sites_c), _f64(x_c)
    si, xi = _f64(sites_i), _f64(x_i)
    nc, ni = int(sc.shape[0]), int(si.shape[0])
    nb = _i32(nbr) if (m > 0 and nc > 0) else None
    lg, se = C.c_double(), C.c_double()
    _check(lib().vecchia_censored_log_cdf(ctx.handle, _ptr(sc) if nc else None, nc, _ptr(nb), int(m),
                                          _ptr(si) if ni else None, ni, make_cov(cov), _ptr(xc) if nc else None,
                                          _ptr(xi) if ni else None, int(N), int(S), C.c_uint64(int(seed)),
                                          float(beta), float(gamma), int(n_nodes), int(precision), C.byref(lg),
                                          C.byref(se)), "vecchia_censored_log_cdf", ctx)
    return lg.value, se.value


def vecchia_log_cdf_unordered(ctx, sites, u, m, cov, N, S, seed=0, precision=MIXED, order="xy", perm_out=None):
    """Order, neighbours and the log-CDF in one call from unordered sites;
    returns (log_p, std_err).  perm_out: optional int32 array of D (host or
    device) that receives the ordering."""
    s, uu = _f64(sites), _f64(u)
    k = ORDER_KINDS.get(order, order) if isinstance(order, str) else int(order)
    lp, se = C.c_double(), C.c_double()
    _check(lib().vecchia_log_cdf_unordered(ctx.handle, _ptr(s), _ptr(uu), s.shape[0], k, int(m), make_cov(cov),
                                           int(N), int(S), C.c_uint64(int(seed)), int(precision), _ptr(perm_out),
                                           C.byref(lp), C.byref(se)), "vecchia_log_cdf_unordered", ctx)
    return lp.value, se.value


def vecchia_mixture_log_cdf(ctx, sites_ordered, nbr, m, cov, x, N, S, seed=0, beta=0.5, gamma=1.0,
                            n_nodes=16, precision=MIXED):
    s, xx = _f64(sites_ordered), _f64(x)
    nb = _i32(nbr) if m > 0 else None
    lg, se = C.c_double(), C.c_double()
    _check(lib().vecchia_mixture_log_cdf(ctx.handle, _ptr(s), s.shape[0], _ptr(nb), int(m), make_cov(cov),
                                         _ptr(xx), int(N), int(S), C.c_uint64(int(seed)), float(beta),
                                         float(gamma), int(n_nodes), int(precision), C.byref(lg),
                                         C.byref(se)), "vecchia_mixture_log_cdf", ctx)
    return lg.value, se.value


def vecchia_log_cdf_noalloc(device, stream, sites_ordered, nbr, m, cov, u, N, S, seed=0,
                            precision=MIXED):
    """The log-CDF with no allocation (scratch in the library's fixed device
    array); device arrays in, (log_p, std_err) out.  No context is used."""
    s, uu = _f64(sites_ordered), _f64(u)
    nb = _i32(nbr) if m > 0 else None
    lp, se = C.c_double(), C.c_double()
    _check(lib().vecchia_log_cdf_noalloc(int(device), _vp(stream or 0), _ptr(s), s.shape[0], _ptr(nb),
                                         int(m), make_cov(cov), _ptr(uu), int(N), int(S),
                                         C.c_uint64(int(seed)), int(precision), C.byref(lp), C.byref(se)),
           "vecchia_log_cdf_noalloc")
    return lp.value, se.value


def vecchia_log_cdf_terms(ctx, sites_ordered, nbr, m, cov, u, N, S, seed=0, precision=MIXED):
    """Returns (log_p, std_err, terms[D], num[D,S], den[D,S]) on the inputs' device."""
    s, uu = _f64(sites_ordered), _f64(u)
    nb = _i32(nbr) if m > 0 else None
    D = s.shape[0]
    tdt = torch.float64 if torch is not None else None
    terms = _empty_like_kind(s, (D,), np.float64, tdt)
    num = _empty_like_kind(s, (D, int(S)), np.float64, tdt)
    den = _empty_like_kind(s, (D, int(S)), np.float64, tdt)
    lp, se = C.c_double(), C.c_double()
    _check(lib().vecchia_log_cdf_terms(ctx.handle, _ptr(s), D, _ptr(nb), int(m), make_cov(cov),
                                       _ptr(uu), int(N), int(S), C.c_uint64(int(seed)),
                                       int(precision), C.byref(lp), C.byref(se), _ptr(terms),
                                       _ptr(num), _ptr(den)), "vecchia_log_cdf_terms", ctx)
    return lp.value, se.value, terms, num, den


def _problem_array(problems):
    n = len(problems)
    arr = (vecchia_problem * n)()
    keep = []
    for i, p in enumerate(problems):
        s, uu = _f64(p["sites"]), _f64(p["u"])
        m = int(p["m"])
        nb = _i32(p["nbr"]) if m > 0 else None
        keep.append((s, uu, nb))
        arr[i] = vecchia_problem(_ptr(s), _ptr(nb), _ptr(uu), s.shape[0], m, int(p["S"]), int(p["N"]),
                                 int(p.get("seed", 0)), make_cov(p["cov"]), int(p.get("group", 0)),
                                 int(p.get("cond_max", 0)))
    return arr, keep


def vecchia_log_cdf_batch(ctx, problems, precision=MIXED):
    """problems: list of dicts with keys sites, nbr, m, cov, u, N, S, seed and
    optionally group, cond_max (arrays all host or all device).  Returns numpy
    arrays (log_p, std_err, status)."""
    n = len(problems)
    arr, keep = _problem_array(problems)
    lp = np.empty(n)
    se = np.empty(n)
    st = np.empty(n, dtype=np.int32)
    _check(lib().vecchia_log_cdf_batch(ctx.handle, arr, n, int(precision), lp.ctypes.data,
                                       se.ctypes.data, st.ctypes.data), "vecchia_log_cdf_batch", ctx)
    return lp, se, st


class Plan:
    """vecchia_plan: a batch kept resident and replayed as a CUDA graph."""

    def __init__(self, ctx, problems, precision=MIXED):
        self.n = len(problems)
        arr, self._keep = _problem_array(problems)  # device arrays must outlive the plan
        self.status = np.empty(self.n, dtype=np.int32)
        h = _vp()
        _check(lib().vecchia_plan_create(ctx.handle, arr, self.n, int(precision), C.byref(h),
                                         self.status.ctypes.data), "vecchia_plan_create", ctx)
        self.handle = h
        self.ctx = ctx

    def run(self, seeds=None, covs=None):
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        cv = None
        if covs is not None:
            cv = (vecchia_cov * self.n)(*[make_cov(c) for c in covs])
        lp = np.empty(self.n)
        se = np.empty(self.n)
        st = np.empty(self.n, dtype=np.int32)
        _check(lib().vecchia_plan_run(self.handle, None if sd is None else sd.ctypes.data,
                                      None if cv is None else C.addressof(cv), lp.ctypes.data,
                                      se.ctypes.data, st.ctypes.data), "vecchia_plan_run", self.ctx)
        return lp, se, st

    def close(self):
        if getattr(self, "handle", None):
            lib().vecchia_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vecchia_plan_create(ctx, problems, precision=MIXED):
    return Plan(ctx, problems, precision)


def vecchia_neighbors_async(ctx, sites_ordered, m, out=None):
    """Queue the neighbour search for device arrays; returns the (not yet
    filled) int32 tensor."""
    s = sites_ordered
    D = s.shape[0]
    nbr = out if out is not None else torch.empty((D, max(int(m), 0)), dtype=torch.int32, device=s.device)
    _check(lib().vecchia_neighbors_async(ctx.handle, _ptr(s), D, int(m), _ptr(nbr) if m > 0 else None),
           "vecchia_neighbors_async", ctx)
    return nbr


def vecchia_result_init(ctx, results, n):
    """results: a device tensor holding n 32-byte result slots."""
    _check(lib().vecchia_result_init(ctx.handle, _ptr(results), int(n)), "vecchia_result_init", ctx)


def make_segment(sites, nbr, u, m, cov, N, S, seed, num, den, result_ptr, site_begin, site_count, group=0):
    prob = vecchia_problem(_ptr(sites), _ptr(nbr) if m > 0 else None, _ptr(u), sites.shape[0], int(m),
                           int(S), int(N), int(seed), make_cov(cov), int(group), 0)
    return vecchia_segment(prob, _ptr(num), _ptr(den), result_ptr, int(site_begin), int(site_count))


def vecchia_partials_async(ctx, segments, precision=MIXED):
    n = len(segments)
    arr = (vecchia_segment * n)(*segments)
    _check(lib().vecchia_partials_async(ctx.handle, arr, n, int(precision)), "vecchia_partials_async", ctx)


def vecchia_reduce_async(ctx, segments):
    n = len(segments)
    arr = (vecchia_segment * n)(*segments)
    _check(lib().vecchia_reduce_async(ctx.handle, arr, n), "vecchia_reduce_async", ctx)


def vecchia_lattice(N, dim):
    g = np.zeros(int(dim), dtype=np.uint32)
    _check(lib().vecchia_lattice(int(N), int(dim), g.ctypes.data if dim > 0 else None),
           "vecchia_lattice")
    return g


def vecchia_shifts(seed, S, dim):
    d = np.zeros((int(S), int(dim)), dtype=np.float64)
    _check(lib().vecchia_shifts(C.c_uint64(int(seed)), int(S), int(dim), d.ctypes.data if d.size else None),
           "vecchia_shifts")
    return d


def vecchia_last_error_site(ctx):
    return lib().vecchia_last_error_site(ctx.handle)


def vecchia_set_tile(ctx, precision, bucket, warps, points, slices, groups):
    _check(lib().vecchia_set_tile(ctx.handle, int(precision), int(bucket), int(warps), int(points),
                                  int(slices), int(groups)), "vecchia_set_tile", ctx)


def vecchia_reset_tiles(ctx):
    _check(lib().vecchia_reset_tiles(ctx.handle), "vecchia_reset_tiles", ctx)


def vecchia_eval_special(ctx, which, x):
    """FP32 special functions of the mixed path on a CUDA float32 tensor (diagnostic)."""
    xx = x.to(torch.float32).contiguous()
    out = torch.empty_like(xx)
    _check(lib().vecchia_eval_special(ctx.handle, int(which), _ptr(xx), xx.numel(), _ptr(out)),
           "vecchia_eval_special", ctx)
    return out


def vecchia_eval_special64(ctx, which, x):
    """FP64 special functions of the FP64 path on a CUDA float64 tensor (diagnostic)."""
    xx = x.to(torch.float64).contiguous()
    out = torch.empty_like(xx)
    _check(lib().vecchia_eval_special64(ctx.handle, int(which), _ptr(xx), xx.numel(), _ptr(out)),
           "vecchia_eval_special64", ctx)
    return out


def vecchia_set_timing(ctx, enable=True):
    _check(lib().vecchia_set_timing(ctx.handle, 1 if enable else 0), "vecchia_set_timing", ctx)


def vecchia_set_full_genz_wait(ctx, limit_ns=0, withhold=False):
    """Wait limit of the tensor-core full-Genz kernel (0 = built-in 2 s) and
    the test switch that makes its copy lane issue nothing."""
    _check(lib().vecchia_set_full_genz_wait(ctx.handle, C.c_uint64(int(limit_ns)), 1 if withhold else 0),
           "vecchia_set_full_genz_wait", ctx)


def vecchia_genz_time_ms(ctx):
    v = C.c_double()
    _check(lib().vecchia_genz_time_ms(ctx.handle, C.byref(v)), "vecchia_genz_time_ms", ctx)
    return v.value
