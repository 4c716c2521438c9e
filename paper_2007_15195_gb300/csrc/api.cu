// api.cu -- the C ABI of libvecchia (include/vecchia.h): context, argument
// checks, device scratch arena, host-side generators (Korobov lattice,
// Philox shifts), host ordering, and the launch sequence of the log-CDF.
#include <omp.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "vk_internal.h"

struct vecchia_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    void* arena = nullptr;
    size_t arena_cap = 0;
    void* host_stage = nullptr;  // pinned
    size_t host_stage_cap = 0;
    void* aux = nullptr;  // device buffer for inputs derived before a batch (kept apart from the arena)
    size_t aux_cap = 0;
    std::map<int64_t, uint32_t*> lattice_dev;  // N -> device [g(32) | gfix(32)]
    int64_t last_error_site = -1;
    vk::GenzTile tile[2][vk::kNumBuckets];
    bool tile_set[2][vk::kNumBuckets] = {{false}};
    bool timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double genz_ms = 0.0;
    // asynchronous calls: two pinned parameter buffers used in turn, each
    // reused only after the upload that last read it has executed
    void* astage[2] = {nullptr, nullptr};
    size_t astage_cap[2] = {0, 0};
    cudaEvent_t astage_ev[2] = {nullptr, nullptr};
    int astage_i = 0;
    // tensor-core full Genz: limit of its progress waits (0 = built-in) and the
    // test switch that makes its copy lane issue nothing
    uint64_t full_wait_ns = 0;
    int full_withhold = 0;
    int* small_dev = nullptr;  // a device int for small reductions (allocated on first use)
};

namespace vk {

int device_sm_count(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 1;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
            v = 1;
        cached[device] = v;
    }
    return cached[device];
}

}  // namespace vk

namespace {

using vk::GenzTile;
using vk::ProbDev;
using vk::ProbResult;

constexpr int kDim = vk::kMaxDim;  // shift-table stride and lattice length

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ensure_arena(vecchia_ctx* c, size_t bytes) {
    if (bytes <= c->arena_cap) return VECCHIA_OK;
    if (c->arena) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->arena);
        c->arena = nullptr;
        c->arena_cap = 0;
    }
    size_t cap = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&c->arena, cap) != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_NOMEM;
    }
    c->arena_cap = cap;
    return VECCHIA_OK;
}

int ensure_aux(vecchia_ctx* c, size_t bytes) {
    if (bytes <= c->aux_cap) return VECCHIA_OK;
    if (c->aux) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->aux);
        c->aux = nullptr;
        c->aux_cap = 0;
    }
    if (cudaMalloc(&c->aux, bytes) != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_NOMEM;
    }
    c->aux_cap = bytes;
    return VECCHIA_OK;
}

int ensure_stage(vecchia_ctx* c, size_t bytes) {
    if (bytes <= c->host_stage_cap) return VECCHIA_OK;
    if (c->host_stage) {
        cudaStreamSynchronize(c->stream);
        cudaFreeHost(c->host_stage);
        c->host_stage = nullptr;
        c->host_stage_cap = 0;
    }
    size_t cap = std::max(bytes, (size_t)1 << 16);
    if (cudaMallocHost(&c->host_stage, cap) != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_NOMEM;
    }
    c->host_stage_cap = cap;
    return VECCHIA_OK;
}

// Bump allocator over a base pointer (device arena or host staging).
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* b) : base((char*)b) {}
    template <class T>
    T* take(size_t count) {
        T* p = (T*)(base ? base + off : nullptr);
        off += al256(sizeof(T) * std::max<size_t>(count, 1));
        return p;
    }
};

// ------------------------- Korobov lattice (host) --------------------------
// The weighted P2 criterion of g_j = a^j mod N over 30 dimensions, weights
// gamma_j = 1/j^2:  P2 = -1 + (1/N) sum_k prod_j (1 + gamma_j 2 pi^2 B2({k g_j/N})),
// B2(x) = x^2 - x + 1/6.  Evaluated in this fixed order of operations.

double p2_of(int64_t N, int64_t a, const std::vector<double>& b2) {
    constexpr int dim = 30;
    const double pi = 3.14159265358979323846;
    const double two_pi_sq = 2.0 * pi * pi;
    int64_t g[dim], r[dim];
    double c[dim];
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
        for (int j = 0; j < dim; ++j) prod *= (1.0 + c[j] * b2[(size_t)r[j]]);
        acc += prod;
        for (int j = 0; j < dim; ++j) {
            r[j] += g[j];
            if (r[j] >= N) r[j] -= N;
        }
    }
    return acc / (double)N - 1.0;
}

int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

std::mutex g_korobov_mu;
std::map<int64_t, int64_t> g_korobov;

int64_t korobov_multiplier(int64_t N) {
    if (N < 4) return 1;
    {
        std::lock_guard<std::mutex> lk(g_korobov_mu);
        auto it = g_korobov.find(N);
        if (it != g_korobov.end()) return it->second;
    }
    std::vector<double> b2((size_t)N);
    for (int64_t r = 0; r < N; ++r) {
        const double x = (double)r / (double)N;
        b2[(size_t)r] = (x * x - x) + (1.0 / 6.0);
    }
    const int64_t amax = N / 2;
    std::vector<double> crit((size_t)amax + 1, INFINITY);
    const int nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            for (int64_t a = 2 + t; a <= amax; a += nt)
                if (gcd64(a, N) == 1) crit[(size_t)a] = p2_of(N, a, b2);
        });
    }
    for (auto& x : th) x.join();
    int64_t best = 1;
    double bv = INFINITY;
    for (int64_t a = 2; a <= amax; ++a) {
        if (crit[(size_t)a] < bv) {
            bv = crit[(size_t)a];
            best = a;
        }
    }
    std::lock_guard<std::mutex> lk(g_korobov_mu);
    g_korobov[N] = best;
    return best;
}

void lattice_host(int64_t N, int dim, uint32_t* g) {
    const int64_t a = korobov_multiplier(N);
    int64_t v = 1 % N;
    for (int j = 0; j < dim; ++j) {
        g[j] = (uint32_t)v;
        v = (v * a) % N;
    }
}

// --------------------------- Philox4x32-10 (host) ---------------------------

void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t m0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t m1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = (uint32_t)m1;
        c[2] = n2;
        c[3] = (uint32_t)m0;
    }
}

// ----------------------------- argument checks ------------------------------

bool cov_ok(const vecchia_cov& c) {
    if (!(c.variance > 0.0) || !(c.range > 0.0) || !(c.nugget >= 0.0)) return false;
    if (!std::isfinite(c.variance) || !std::isfinite(c.range) || !std::isfinite(c.nugget)) return false;
    if (c.kind == VECCHIA_COV_EXPONENTIAL) return true;
    if (c.kind == VECCHIA_COV_MATERN) return c.nu == 0.5 || c.nu == 1.5 || c.nu == 2.5;
    if (c.kind == VECCHIA_COV_ANISO_EXP)
        return std::isfinite(c.angle) && std::isfinite(c.aspect) && c.aspect > 0.0;
    return false;
}

void set_cov(ProbDev& d, const vecchia_cov& c) {
    d.variance = c.variance;
    d.range = c.range;
    d.nu = c.nu;
    d.nugget = c.nugget;
    d.cov_kind = c.kind;
    d.cos_a = (c.kind == VECCHIA_COV_ANISO_EXP) ? std::cos(c.angle) : 1.0;
    d.sin_a = (c.kind == VECCHIA_COV_ANISO_EXP) ? std::sin(c.angle) : 0.0;
    d.aspect = (c.kind == VECCHIA_COV_ANISO_EXP) ? c.aspect : 1.0;
}

int check_problem(const vecchia_problem& p) {
    if (p.D < 1 || p.D > INT_MAX / 2 || !p.sites || !p.u) return VECCHIA_ERR_ARG;
    if (p.m < 0 || p.group < 0 || p.cond_max < 0 || p.cond_max > p.m) return VECCHIA_ERR_ARG;
    if (p.m > VECCHIA_MAX_M || vk::max_term_dim(p.m, p.group) > VECCHIA_MAX_M + 1)
        return VECCHIA_ERR_UNSUPPORTED;
    if (p.m > 0 && !p.nbr) return VECCHIA_ERR_ARG;
    if (p.N < 1 || p.N > INT_MAX) return VECCHIA_ERR_ARG;
    if (p.S < 2 || p.S > VECCHIA_MAX_S) return VECCHIA_ERR_ARG;
    if (!cov_ok(p.cov)) return VECCHIA_ERR_ARG;
    return VECCHIA_OK;
}

uint32_t* lattice_for(vecchia_ctx* c, int64_t N) {
    auto it = c->lattice_dev.find(N);
    if (it != c->lattice_dev.end()) return it->second;
    uint32_t h[2 * kDim];
    lattice_host(N, kDim, h);
    for (int j = 0; j < kDim; ++j)  // round(g 2^32 / N): exact when N is a power of two
        h[kDim + j] = (uint32_t)((((uint64_t)h[j] << 32) + (uint64_t)N / 2) / (uint64_t)N);
    uint32_t* d = nullptr;
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    c->lattice_dev[N] = d;
    return d;
}

// Built-in tile (measured on the 50x50 grid): mixed blocks of up to 32
// variables run two points per lane (one vote per step for both), 4 warps up
// to 21 variables and 8 above; FP64 one point, 4 warps.  Shift groups (a power
// of two, so S = 2^k splits evenly) until a launch has ~2048 CTA items, never
// fewer shifts per item than warps (a warp without a unit idles); ~4096 items
// for blocks of up to 16 variables, which fit more CTAs per SM.  Blocks
// above 32 variables: 8 warps, one point per lane, every shift of a term in
// one item, so the one-warp Cholesky of up to 64 variables is shared by the
// most work.
GenzTile default_tile(bool mixed, int64_t total_sites, int max_S, int bucket) {
    GenzTile t;
    const int dmax = vk::kDmaxBuckets[bucket];
    if (dmax > 32) {
        t.warps = 8;
        t.points = 1;
        t.slices = 1;
        t.groups = 1;
        return t;
    }
    t.warps = (mixed && dmax > 21) ? 8 : 4;
    t.points = mixed ? 2 : 1;
    t.slices = 1;
    // small blocks fit more CTAs per SM: they want more items
    const int64_t target = dmax <= 16 ? 4096 : 2048;
    int g = 1;
    while (g < max_S && (int64_t)g * total_sites < target && max_S / (2 * g) >= t.warps) g *= 2;
    t.groups = g;
    return t;
}

// ------------------------------ the pipeline --------------------------------
// A batch of n problems: validation and buckets (Batch, prepare), a layout of
// one device arena and one host parameter blob, and the launch sequence
// (enqueue): blob upload, result init, shift tables, Genz per bucket (largest
// blocks first), the log-space re-evaluation of flagged terms (mixed), the
// two log-sum passes, the result download.  vecchia_log_cdf* run it once on
// the context's arena; a plan owns its buffers and replays it as a CUDA graph.

constexpr int NB = vk::kNumBuckets;

struct Batch {
    int n = 0;
    bool mixed = false, host_in = false, terms_host = false;
    std::vector<vecchia_problem> probs;
    std::vector<int> ok;
    int64_t total_sites = 0, fb_cap = 0, max_slices = 0;  // total_sites: terms of all problems
    int64_t total_shift_rows = 0;
    int max_S[NB] = {0};
    int max_S_all = 0, max_bucket = 0;
    int64_t bucket_sites[NB] = {0};
    int bucket_segs[NB] = {0};
    GenzTile tiles[NB];
    std::vector<int> bucket_of;
    std::vector<uint32_t*> lat;
    // device arena offsets
    std::vector<size_t> o_sites, o_nbr, o_u, o_num, o_den;
    size_t o_means = 0, o_delta = 0, o_dfix = 0, o_fbcount = 0, o_fbitems = 0, o_terms_out = 0, o_blob = 0;
    size_t arena_bytes = 0;
    // host blob offsets (the blob is copied to o_blob)
    size_t b_probs = 0, b_results = 0, b_seeds = 0, b_S = 0, b_off = 0, b_moff = 0, b_tptr = 0;
    size_t b_segp[NB] = {0}, b_segb[NB] = {0};
    size_t blob_bytes = 0;
};

// Validation, buckets, tiles, lattice tables and the layout; allocates nothing
// but the per-N lattice tables of the context.  status[] gets per-problem codes.
int prepare(vecchia_ctx* c, const vecchia_problem* probs, int n, int precision, int32_t* status,
            bool with_terms, bool terms_host, Batch& B) {
    if (precision != VECCHIA_FP64 && precision != VECCHIA_MIXED) return VECCHIA_ERR_ARG;
    B.n = n;
    B.mixed = precision == VECCHIA_MIXED;
    B.probs.assign(probs, probs + n);
    B.ok.assign(n, 0);
    int n_ok = 0;
    for (int i = 0; i < n; ++i) {
        status[i] = check_problem(probs[i]);
        B.ok[i] = status[i] == VECCHIA_OK;
        n_ok += B.ok[i];
    }
    if (n_ok == 0) return VECCHIA_OK;
    B.host_in = !is_device_ptr(probs[0].sites);
    if (B.host_in) {  // a host problem with NaN thresholds is an argument error
        for (int i = 0; i < n; ++i) {
            if (!B.ok[i]) continue;
            for (int64_t k = 0; k < probs[i].D; ++k) {
                if (!std::isfinite(probs[i].u[k])) {
                    status[i] = VECCHIA_ERR_ARG;
                    B.ok[i] = 0;
                    break;
                }
            }
        }
    }
    B.bucket_of.assign(n, -1);
    for (int i = 0; i < n; ++i) {
        if (!B.ok[i]) continue;
        const int b = vk::bucket_of(vk::max_term_dim(probs[i].m, probs[i].group, probs[i].cond_max));
        const int64_t T = vk::n_terms_of(probs[i].D, probs[i].group);
        B.bucket_of[i] = b;
        B.bucket_sites[b] += T;
        B.bucket_segs[b] += 1;
        B.max_S[b] = std::max(B.max_S[b], probs[i].S);
        B.max_S_all = std::max(B.max_S_all, probs[i].S);
        B.max_bucket = std::max(B.max_bucket, b);
        B.total_sites += T;
        B.total_shift_rows += probs[i].S;
        B.max_slices = std::max(B.max_slices, vk::logsum_slices(T));
    }
    int max_groups = 1;
    for (int b = 0; b < NB; ++b) {
        B.tiles[b] = c->tile_set[B.mixed][b] ? c->tile[B.mixed][b]
                                             : default_tile(B.mixed, B.total_sites, std::max(B.max_S[b], 2), b);
        max_groups = std::max(max_groups, B.tiles[b].groups);
    }
    B.fb_cap = B.mixed ? B.total_sites * max_groups + vk::genz_items_slack(vk::device_sm_count(c ? c->device : 0)) : 0;
    B.lat.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        if (!B.ok[i]) continue;
        B.lat[i] = lattice_for(c, probs[i].N);
        if (!B.lat[i]) return VECCHIA_ERR_NOMEM;
    }
    // device arena
    Carve dv(nullptr);
    B.o_sites.assign(n, 0);
    B.o_nbr.assign(n, 0);
    B.o_u.assign(n, 0);
    B.o_num.assign(n, 0);
    B.o_den.assign(n, 0);
    int64_t logsum_doubles = 0;
    for (int i = 0; i < n; ++i) {
        if (!B.ok[i]) continue;
        const auto& p = probs[i];
        const int64_t T = vk::n_terms_of(p.D, p.group);
        if (B.host_in) {
            B.o_sites[i] = dv.off;
            dv.take<double>(2 * p.D);
            B.o_nbr[i] = dv.off;
            dv.take<int32_t>((size_t)T * std::max(p.m, 1));
            B.o_u[i] = dv.off;
            dv.take<double>(p.D);
        }
        B.o_num[i] = dv.off;
        dv.take<double>((size_t)T * p.S);
        B.o_den[i] = dv.off;
        dv.take<double>((size_t)T * p.S);
        logsum_doubles += vk::logsum_scratch(T, p.S);
    }
    B.o_means = dv.off;
    dv.take<double>(logsum_doubles);
    B.o_delta = dv.off;
    dv.take<double>((size_t)B.total_shift_rows * kDim);
    B.o_dfix = dv.off;
    dv.take<uint32_t>((size_t)B.total_shift_rows * kDim);
    B.o_fbcount = dv.off;
    dv.take<int>(1);
    B.o_fbitems = dv.off;
    dv.take<int2>((size_t)std::max<int64_t>(B.fb_cap, 1));
    B.terms_host = with_terms && terms_host;
    B.o_terms_out = dv.off;
    if (B.terms_host) dv.take<double>(B.total_sites);
    // parameter blob
    Carve hb(nullptr);
    B.b_probs = hb.off;
    hb.take<ProbDev>(n);
    B.b_results = hb.off;
    hb.take<ProbResult>(n);
    B.b_seeds = hb.off;
    hb.take<uint64_t>(n);
    B.b_S = hb.off;
    hb.take<int32_t>(n);
    B.b_off = hb.off;
    hb.take<int64_t>(n);
    B.b_moff = hb.off;
    hb.take<int64_t>(n);
    B.b_tptr = hb.off;
    hb.take<double*>(n);
    for (int b = 0; b < NB; ++b) {
        B.b_segp[b] = hb.off;
        hb.take<int>(B.bucket_segs[b] + 1);
        B.b_segb[b] = hb.off;
        hb.take<int2>(std::max(B.bucket_segs[b], 1));
    }
    B.blob_bytes = hb.off;
    B.o_blob = dv.off;
    dv.take<char>(B.blob_bytes);
    B.arena_bytes = dv.off;
    return VECCHIA_OK;
}

// The host blob: problem descriptors (device pointers into A), seeds, offsets,
// segments.  terms: device array of the single problem's terms (or nullptr).
void fill_blob(const Batch& B, char* A, char* H, double* terms) {
    ProbDev* hp = (ProbDev*)(H + B.b_probs);
    uint64_t* hseeds = (uint64_t*)(H + B.b_seeds);
    int32_t* hS = (int32_t*)(H + B.b_S);
    int64_t* hoff = (int64_t*)(H + B.b_off);
    int64_t* hmoff = (int64_t*)(H + B.b_moff);
    double** htp = (double**)(H + B.b_tptr);
    int64_t moff = 0, soff = 0;
    for (int i = 0; i < B.n; ++i) {
        const auto& p = B.probs[i];
        ProbDev& d = hp[i];
        std::memset(&d, 0, sizeof(d));
        hseeds[i] = p.seed;
        hS[i] = B.ok[i] ? p.S : 0;
        hoff[i] = soff;
        hmoff[i] = moff;
        htp[i] = nullptr;
        if (!B.ok[i]) continue;
        soff += (int64_t)p.S * kDim;
        d.sites = B.host_in ? (const double*)(A + B.o_sites[i]) : p.sites;
        d.nbr = B.host_in ? (const int32_t*)(A + B.o_nbr[i]) : p.nbr;
        d.u = B.host_in ? (const double*)(A + B.o_u[i]) : p.u;
        d.num = (double*)(A + B.o_num[i]);
        d.den = (double*)(A + B.o_den[i]);
        d.g = B.lat[i];
        d.gfix = B.lat[i] + kDim;
        d.delta = (const double*)(A + B.o_delta) + hoff[i];
        d.dfix = (const uint32_t*)(A + B.o_dfix) + hoff[i];
        d.D = p.D;
        d.n_terms = vk::n_terms_of(p.D, p.group);
        d.N = p.N;
        set_cov(d, p.cov);
        d.m = p.m;
        d.group = p.group;
        d.S = p.S;
        d.dim = kDim;
        if (terms) htp[i] = B.terms_host ? (double*)(A + B.o_terms_out) : terms;
        moff += vk::logsum_scratch(d.n_terms, p.S);
    }
    for (int b = 0; b < NB; ++b) {
        int* sp = (int*)(H + B.b_segp[b]);
        int2* sb = (int2*)(H + B.b_segb[b]);
        int k = 0, run = 0;
        for (int i = 0; i < B.n; ++i) {
            if (!B.ok[i] || B.bucket_of[i] != b) continue;
            sp[k] = run;
            sb[k] = make_int2(i, 0);
            run += (int)vk::n_terms_of(B.probs[i].D, B.probs[i].group);
            ++k;
        }
        sp[k] = run;
    }
}

cudaError_t stage_inputs(const Batch& B, char* A, cudaStream_t s) {
    if (!B.host_in) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < B.n && e == cudaSuccess; ++i) {
        if (!B.ok[i]) continue;
        const auto& p = B.probs[i];
        e = cudaMemcpyAsync(A + B.o_sites[i], p.sites, sizeof(double) * 2 * p.D, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && p.m > 0)
            e = cudaMemcpyAsync(A + B.o_nbr[i], p.nbr, sizeof(int32_t) * vk::n_terms_of(p.D, p.group) * p.m,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(A + B.o_u[i], p.u, sizeof(double) * p.D, cudaMemcpyHostToDevice, s);
    }
    return e;
}

// The device sequence (capturable): blob upload ... result download into H.
cudaError_t enqueue(const Batch& B, char* A, char* H, cudaStream_t s, bool with_terms, vecchia_ctx* c) {
    char* blob_dev = A + B.o_blob;
    cudaError_t e = cudaMemcpyAsync(blob_dev, H, B.blob_bytes, cudaMemcpyHostToDevice, s);
    ProbDev* probs_d = (ProbDev*)(blob_dev + B.b_probs);
    ProbResult* res_d = (ProbResult*)(blob_dev + B.b_results);
    int* fbc = (int*)(A + B.o_fbcount);
    int2* fbi = (int2*)(A + B.o_fbitems);
    if (e == cudaSuccess) e = vk::launch_init_results(res_d, B.n, fbc, s);
    if (e == cudaSuccess)
        e = vk::launch_shifts((const uint64_t*)(blob_dev + B.b_seeds), (const int32_t*)(blob_dev + B.b_S),
                              (const int64_t*)(blob_dev + B.b_off), B.n, kDim, (double*)(A + B.o_delta),
                              (uint32_t*)(A + B.o_dfix), s);
    if (c && c->timing && e == cudaSuccess) e = cudaEventRecord(c->ev0, s);
    for (int b = NB - 1; b >= 0 && e == cudaSuccess; --b) {  // largest blocks first
        if (!B.bucket_sites[b]) continue;
        e = vk::launch_genz(b, B.mixed, B.tiles[b], probs_d, (const int*)(blob_dev + B.b_segp[b]),
                            (const int2*)(blob_dev + B.b_segb[b]), B.bucket_segs[b], (int)B.bucket_sites[b],
                            res_d, fbc, fbi, B.max_S[b], (int)B.fb_cap, s);
    }
    if (c && c->timing && e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
    if (B.mixed && e == cudaSuccess)
        e = vk::launch_genz_fallback(B.max_bucket, probs_d, fbc, fbi, (int)B.fb_cap, res_d, B.max_S_all, s);
    if (e == cudaSuccess)
        e = vk::launch_logsum(probs_d, B.n, (int)B.max_slices, res_d,
                              with_terms ? (double* const*)(blob_dev + B.b_tptr) : nullptr,
                              (double*)(A + B.o_means), (const int64_t*)(blob_dev + B.b_moff), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(H + B.b_results, res_d, sizeof(ProbResult) * B.n, cudaMemcpyDeviceToHost, s);
    return e;
}

void collect(const Batch& B, const char* H, double* log_p, double* std_err, int32_t* status,
             int64_t* last_error_site) {
    const ProbResult* hres = (const ProbResult*)(H + B.b_results);
    for (int i = 0; i < B.n; ++i) {
        log_p[i] = NAN;
        std_err[i] = NAN;
        if (!B.ok[i]) continue;
        status[i] = hres[i].status;
        if (hres[i].status == VECCHIA_OK) {
            log_p[i] = hres[i].log_p;
            std_err[i] = hres[i].std_err;
        } else if (hres[i].bad_site != LLONG_MAX && *last_error_site < 0) {
            *last_error_site = hres[i].bad_site;
        }
    }
}

// lr_V, lr_k, lr_scale (one per problem): a low-rank correction of every
// problem's covariance (device V, nc x lr_k), for conditional laws.
int run_problems(vecchia_ctx* c, const vecchia_problem* probs, int n, int precision,
                 double* log_p, double* std_err, int32_t* status, double* terms, double* num,
                 double* den, const double* lr_V = nullptr, int lr_k = 0, const double* lr_scale = nullptr) {
    if (!c || !probs || n < 1 || !log_p || !std_err || !status) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    c->last_error_site = -1;
    for (int i = 0; i < n; ++i) {
        log_p[i] = NAN;
        std_err[i] = NAN;
    }
    Batch B;
    const bool terms_host = terms && !is_device_ptr(terms);
    int st = prepare(c, probs, n, precision, status, terms != nullptr, terms_host, B);
    if (st != VECCHIA_OK) return st;
    int n_ok = 0;
    for (int i = 0; i < n; ++i) n_ok += B.ok[i];
    if (n_ok == 0) return n == 1 ? status[0] : VECCHIA_OK;
    st = ensure_arena(c, B.arena_bytes);
    if (st != VECCHIA_OK) return st;
    st = ensure_stage(c, B.blob_bytes);
    if (st != VECCHIA_OK) return st;
    char* A = (char*)c->arena;
    char* H = (char*)c->host_stage;
    fill_blob(B, A, H, terms);
    if (lr_k > 0) {
        ProbDev* hp = (ProbDev*)(H + B.b_probs);
        for (int i = 0; i < n; ++i) {
            hp[i].lr_V = lr_V;
            hp[i].lr_k = lr_k;
            hp[i].lr_scale = lr_scale[i];
        }
    }
    const cudaStream_t s = c->stream;
    cudaError_t e = stage_inputs(B, A, s);
    if (e == cudaSuccess) e = enqueue(B, A, H, s, terms != nullptr, c);
    if (n == 1 && B.ok[0] && e == cudaSuccess) {
        const auto& p = probs[0];
        const int64_t T = vk::n_terms_of(p.D, p.group);
        if (B.terms_host)
            e = cudaMemcpyAsync(terms, A + B.o_terms_out, sizeof(double) * T, cudaMemcpyDefault, s);
        if (num && e == cudaSuccess)
            e = cudaMemcpyAsync(num, A + B.o_num[0], sizeof(double) * T * p.S, cudaMemcpyDefault, s);
        if (den && e == cudaSuccess)
            e = cudaMemcpyAsync(den, A + B.o_den[0], sizeof(double) * T * p.S, cudaMemcpyDefault, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    if (c->timing) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->genz_ms = ms;
    }
    collect(B, H, log_p, std_err, status, &c->last_error_site);
    return n == 1 ? status[0] : VECCHIA_OK;
}

// ------------------------------ plans (graphs) ------------------------------

}  // namespace

struct vecchia_plan {
    vecchia_ctx* c = nullptr;
    Batch B;
    char* A = nullptr;  // device buffer owned by the plan
    char* H = nullptr;  // pinned parameter blob owned by the plan
    cudaStream_t stream = nullptr;
    cudaEvent_t ready = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void plan_free(vecchia_plan* P) {
    if (!P) return;
    if (P->stream) cudaStreamSynchronize(P->stream);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->ready) cudaEventDestroy(P->ready);
    if (P->stream) cudaStreamDestroy(P->stream);
    if (P->A) cudaFree(P->A);
    if (P->H) cudaFreeHost(P->H);
    delete P;
}

// ------------------------- asynchronous segment calls ------------------------

// A pinned parameter buffer for an asynchronous call, safe to overwrite now.
char* async_stage(vecchia_ctx* c, size_t bytes, int* which) {
    const int k = c->astage_i;
    c->astage_i ^= 1;
    if (cudaEventSynchronize(c->astage_ev[k]) != cudaSuccess) cudaGetLastError();
    if (c->astage_cap[k] < bytes) {
        if (c->astage[k]) cudaFreeHost(c->astage[k]);
        c->astage[k] = nullptr;
        c->astage_cap[k] = 0;
        const size_t cap = std::max(bytes, (size_t)1 << 16);
        if (cudaMallocHost(&c->astage[k], cap) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c->astage_cap[k] = cap;
    }
    *which = k;
    return (char*)c->astage[k];
}

bool segment_ok(const vecchia_segment& g) {
    return check_problem(g.prob) == VECCHIA_OK && g.num && g.den && g.result && g.site_begin >= 0 &&
           g.site_count >= 0 && g.site_begin + g.site_count <= vk::n_terms_of(g.prob.D, g.prob.group);
}

void fill_probdev(ProbDev& d, const vecchia_segment& g, uint32_t* lat, char* A, size_t o_delta,
                  size_t o_dfix, int64_t off) {
    std::memset(&d, 0, sizeof(d));
    const auto& p = g.prob;
    d.sites = p.sites;
    d.nbr = p.nbr;
    d.u = p.u;
    d.num = g.num;
    d.den = g.den;
    d.g = lat;
    d.gfix = lat ? lat + kDim : nullptr;
    d.delta = (const double*)(A + o_delta) + off;
    d.dfix = (const uint32_t*)(A + o_dfix) + off;
    d.D = p.D;
    d.n_terms = vk::n_terms_of(p.D, p.group);
    d.N = p.N;
    set_cov(d, p.cov);
    d.m = p.m;
    d.group = p.group;
    d.S = p.S;
    d.dim = kDim;
    d.res = (ProbResult*)g.result;
}

// ----------------------- scale-mixture CDF (Sec. 4) -------------------------

// Gauss-Legendre rule on [0, 1]: Newton's method on the Legendre polynomial
// P_n from the Chebyshev-like first guesses, weights 2/((1-x^2) P_n'(x)^2)
// (Golub & Welsch give the same rule; this is the classical root iteration).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {  // P_k(z) by the three-term recurrence
                const double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        const double wt = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = 0.5 * (1.0 - z);
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[i] = w[n - 1 - i] = 0.5 * wt;
    }
}

// r = F_R^{-1}(v) for F_R(r) = 1 - exp(-gamma (r^beta - 1)/beta), r >= 1
// (beta > 0), and its beta -> 0 limit F_R(r) = 1 - r^(-gamma), written in
// terms of L = -log(1 - v) >= 0.
double mixing_radius(double L, double beta, double gamma) {
    if (beta > 0.0) return std::pow(1.0 + beta * L / gamma, 1.0 / beta);
    return std::exp(L / gamma);
}

// Nodes r_q and weights w_q of int_0^inf h(r) dF_R(r) = int_0^1 h(F_R^{-1}(v)) dv.
// F_R^{-1} is singular at v = 1, so v = 1 - (1 - t)^4 (dv = 4 (1 - t)^3 dt)
// flattens the integrand there before the Gauss-Legendre rule in t:
// L = -log(1 - v) = -4 log(1 - t).
void mixture_nodes(int n, double beta, double gamma, std::vector<double>& r, std::vector<double>& w) {
    std::vector<double> t;
    gauss_legendre01(n, t, w);
    r.assign(n, 0.0);
    for (int q = 0; q < n; ++q) {
        const double omt = 1.0 - t[q];
        w[q] *= 4.0 * omt * omt * omt;
        r[q] = mixing_radius(-4.0 * std::log1p(-t[q]), beta, gamma);
    }
}

// ------------------------------ host ordering ------------------------------

void quantize_host(const double* s, int64_t D, std::vector<int64_t>& q) {
    q.assign(2 * (size_t)D, 0);
    double x0 = s[0], x1 = s[0], y0 = s[1], y1 = s[1];
    for (int64_t i = 1; i < D; ++i) {
        x0 = std::min(x0, s[2 * i]);
        x1 = std::max(x1, s[2 * i]);
        y0 = std::min(y0, s[2 * i + 1]);
        y1 = std::max(y1, s[2 * i + 1]);
    }
    const double ex = x1 - x0, ey = y1 - y0;
    const double ext = ex > ey ? ex : ey;
    if (!(ext > 0.0)) return;
    const double c = 1073741824.0 / ext;
    for (int64_t i = 0; i < D; ++i) {
        const double tx = s[2 * i] - x0;
        const double ty = s[2 * i + 1] - y0;
        q[2 * (size_t)i] = (int64_t)std::floor(tx * c);
        q[2 * (size_t)i + 1] = (int64_t)std::floor(ty * c);
    }
}

void order_maxmin(const double* s, int64_t D, int32_t* perm) {
    std::vector<int64_t> q;
    quantize_host(s, D, q);
    int64_t qxm = 0, qym = 0;
    for (int64_t i = 0; i < D; ++i) {
        qxm = std::max(qxm, q[2 * i]);
        qym = std::max(qym, q[2 * i + 1]);
    }
    int64_t first = 0, bestc = -1;
    for (int64_t i = 0; i < D; ++i) {
        const int64_t dx = 2 * q[2 * i] - qxm, dy = 2 * q[2 * i + 1] - qym;
        const int64_t v = dx * dx + dy * dy;
        if (bestc < 0 || v < bestc) {
            bestc = v;
            first = i;
        }
    }
    std::vector<int64_t> mind((size_t)D, LLONG_MAX);
    std::vector<char> chosen((size_t)D, 0);
    perm[0] = (int32_t)first;
    chosen[(size_t)first] = 1;
    const int T = D < 4096 ? 1 : std::max(1, std::min(omp_get_max_threads(), 64));
    std::vector<int64_t> tv(T), ti(T);
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t lo = D * t / T, hi = D * (t + 1) / T;
        for (int64_t pos = 1; pos < D; ++pos) {
            const int64_t last = perm[pos - 1];
            const int64_t lx = q[2 * last], ly = q[2 * last + 1];
            int64_t bv = -1, bi = -1;
            for (int64_t i = lo; i < hi; ++i) {
                if (chosen[(size_t)i]) continue;
                const int64_t dx = q[2 * i] - lx, dy = q[2 * i + 1] - ly;
                const int64_t v = std::min(mind[(size_t)i], dx * dx + dy * dy);
                mind[(size_t)i] = v;
                if (v > bv) {
                    bv = v;
                    bi = i;
                }
            }
            tv[t] = bv;
            ti[t] = bi;
#pragma omp barrier
#pragma omp single
            {
                int64_t best = -1, besti = -1;
                for (int k = 0; k < T; ++k)
                    if (tv[k] > best) {  // chunks ascend, so ties keep the smaller index
                        best = tv[k];
                        besti = ti[k];
                    }
                perm[pos] = (int32_t)besti;
                chosen[(size_t)besti] = 1;
            }
        }
    }
}

}  // namespace

// =============================== C ABI ======================================

extern "C" {

const char* vecchia_strerror(int status) {
    switch (status) {
        case VECCHIA_OK: return "ok";
        case VECCHIA_ERR_ARG: return "invalid argument";
        case VECCHIA_ERR_CUDA: return "CUDA runtime error";
        case VECCHIA_ERR_NOMEM: return "out of memory";
        case VECCHIA_ERR_NOT_PD: return "covariance block not positive definite";
        case VECCHIA_ERR_NONFINITE: return "non-finite result";
        case VECCHIA_ERR_TIMEOUT: return "device wait timed out";
        case VECCHIA_ERR_UNSUPPORTED: return "outside this build's limits";
        default: return "unknown status";
    }
}

int vecchia_create(vecchia_ctx** ctx, int device, void* cuda_stream) {
    if (!ctx) return VECCHIA_ERR_ARG;
    *ctx = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    if (device < 0 || device >= n) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    vecchia_ctx* c = new (std::nothrow) vecchia_ctx();
    if (!c) return VECCHIA_ERR_NOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->astage_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->astage_ev[1], cudaEventDisableTiming) != cudaSuccess) {
        delete c;
        return VECCHIA_ERR_CUDA;
    }
    *ctx = c;
    return VECCHIA_OK;
}

int vecchia_destroy(vecchia_ctx* c) {
    if (!c) return VECCHIA_ERR_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->arena) cudaFree(c->arena);
    if (c->aux) cudaFree(c->aux);
    if (c->small_dev) cudaFree(c->small_dev);
    if (c->host_stage) cudaFreeHost(c->host_stage);
    for (auto& kv : c->lattice_dev) cudaFree(kv.second);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (int k = 0; k < 2; ++k) {
        if (c->astage[k]) cudaFreeHost(c->astage[k]);
        if (c->astage_ev[k]) cudaEventDestroy(c->astage_ev[k]);
    }
    delete c;
    return VECCHIA_OK;
}

int vecchia_set_stream(vecchia_ctx* c, void* cuda_stream) {
    if (!c) return VECCHIA_ERR_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return VECCHIA_OK;
}

int64_t vecchia_last_error_site(const vecchia_ctx* c) { return c ? c->last_error_site : -1; }

int vecchia_lattice(int64_t N, int dim, uint32_t* g) {
    if (N < 1 || N > INT_MAX || dim < 0 || (dim > 0 && !g)) return VECCHIA_ERR_ARG;
    lattice_host(N, dim, g);
    return VECCHIA_OK;
}

int vecchia_shifts(uint64_t seed, int S, int dim, double* delta) {
    if (S < 0 || dim < 0 || ((int64_t)S * dim > 0 && !delta)) return VECCHIA_ERR_ARG;
    for (int s = 0; s < S; ++s) {
        for (int j = 0; j < dim; ++j) {
            uint32_t c[4] = {(uint32_t)s, (uint32_t)j, 0x51A7u, 0u};
            philox_host(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
            const uint64_t M = ((uint64_t)(c[0] >> 5) << 26) | (uint64_t)(c[1] >> 6);
            delta[(size_t)s * dim + j] = (double)M * 0x1p-53;
        }
    }
    return VECCHIA_OK;
}

int vecchia_order(vecchia_ctx* c, const double* sites, int64_t D, int kind, int32_t* perm) {
    if (!sites || !perm || D < 1 || D > INT_MAX) return VECCHIA_ERR_ARG;
    if (kind != VECCHIA_ORDER_XY && kind != VECCHIA_ORDER_MAXMIN && kind != VECCHIA_ORDER_IDENTITY)
        return VECCHIA_ERR_ARG;
    // with no context both arrays are host memory and the ordering runs on the host
    const bool dev_in = c && is_device_ptr(sites), dev_out = c && is_device_ptr(perm);
    if (c && (dev_in || dev_out) && cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    if (c && kind == VECCHIA_ORDER_XY && dev_in && dev_out && D <= vk::kOrderXyDeviceMax) {
        // XY on the device: each site's rank counts the smaller (x, y, index) keys
        int st = ensure_arena(c, vk::order_xy_scratch_bytes(D));
        if (st != VECCHIA_OK) return st;
        const cudaError_t e = vk::launch_order_xy(sites, D, perm, c->arena, c->stream);
        if (e != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
            cudaGetLastError();
            return VECCHIA_ERR_CUDA;
        }
        return VECCHIA_OK;
    }
    if (c && kind == VECCHIA_ORDER_MAXMIN) {  // exact maxmin on the device
        if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
        Carve dv(nullptr);
        const size_t o_s = dv.off;
        if (!dev_in) dv.take<double>(2 * D);
        const size_t o_p = dv.off;
        if (!dev_out) dv.take<int32_t>(D);
        const size_t o_scr = dv.off;
        dv.take<char>(vk::maxmin_scratch_bytes(D));
        int st = ensure_arena(c, dv.off);
        if (st != VECCHIA_OK) return st;
        char* A = (char*)c->arena;
        const double* sd = dev_in ? sites : (const double*)(A + o_s);
        int32_t* pd = dev_out ? perm : (int32_t*)(A + o_p);
        cudaError_t e = cudaSuccess;
        if (!dev_in) e = cudaMemcpyAsync(A + o_s, sites, sizeof(double) * 2 * D, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = vk::launch_maxmin(sd, D, pd, A + o_scr, c->stream);
        if (e == cudaSuccess && !dev_out)
            e = cudaMemcpyAsync(perm, pd, sizeof(int32_t) * D, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return VECCHIA_ERR_CUDA;
        }
        return VECCHIA_OK;
    }
    std::vector<double> hs;
    const double* s = sites;
    if (dev_in) {
        hs.resize(2 * (size_t)D);
        if (cudaMemcpyAsync(hs.data(), sites, sizeof(double) * 2 * D, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return VECCHIA_ERR_CUDA;
        s = hs.data();
    }
    std::vector<int32_t> p((size_t)D);
    for (int64_t i = 0; i < D; ++i) p[(size_t)i] = (int32_t)i;
    if (kind == VECCHIA_ORDER_XY) {
        std::sort(p.begin(), p.end(), [s](int32_t a, int32_t b) {
            if (s[2 * a] != s[2 * b]) return s[2 * a] < s[2 * b];
            if (s[2 * a + 1] != s[2 * b + 1]) return s[2 * a + 1] < s[2 * b + 1];
            return a < b;
        });
    } else if (kind == VECCHIA_ORDER_MAXMIN) {
        order_maxmin(s, D, p.data());
    }
    if (dev_out) {
        if (cudaMemcpyAsync(perm, p.data(), sizeof(int32_t) * D, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return VECCHIA_ERR_CUDA;
    } else {
        std::memcpy(perm, p.data(), sizeof(int32_t) * D);
    }
    return VECCHIA_OK;
}

int vecchia_apply_order(vecchia_ctx* c, const int32_t* perm, const double* sites, const double* u,
                        int64_t D, double* sites_out, double* u_out) {
    if (!perm || !sites || !sites_out || D < 1 || D > INT_MAX || (u && !u_out)) return VECCHIA_ERR_ARG;
    if ((const void*)sites == (void*)sites_out || (u && (const void*)u == (void*)u_out)) return VECCHIA_ERR_ARG;
    const bool dev = c && is_device_ptr(sites);
    if (dev) {
        if (!is_device_ptr(perm) || !is_device_ptr(sites_out) || (u && (!is_device_ptr(u) || !is_device_ptr(u_out))))
            return VECCHIA_ERR_ARG;
        if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
        if (ensure_arena(c, 256) != VECCHIA_OK) return VECCHIA_ERR_NOMEM;
        int* bad = (int*)c->arena;
        int hbad = 0;
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = vk::launch_gather(perm, sites, u, D, sites_out, u_out, bad, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return VECCHIA_ERR_CUDA;
        }
        return hbad ? VECCHIA_ERR_ARG : VECCHIA_OK;
    }
    for (int64_t k = 0; k < D; ++k) {
        const int32_t j = perm[k];
        if (j < 0 || j >= D) return VECCHIA_ERR_ARG;
        sites_out[2 * k] = sites[2 * (int64_t)j];
        sites_out[2 * k + 1] = sites[2 * (int64_t)j + 1];
        if (u) u_out[k] = u[j];
    }
    return VECCHIA_OK;
}

int vecchia_log_cdf_unordered(vecchia_ctx* c, const double* sites, const double* u, int64_t D, int order_kind,
                              int m, vecchia_cov cov, int64_t N, int S, uint64_t seed, int precision,
                              int32_t* perm_out, double* log_p, double* std_err) {
    if (!c || !sites || !u || !log_p || !std_err || D < 1 || D > INT_MAX / 2 || m < 0) return VECCHIA_ERR_ARG;
    if (order_kind != VECCHIA_ORDER_XY && order_kind != VECCHIA_ORDER_MAXMIN && order_kind != VECCHIA_ORDER_IDENTITY)
        return VECCHIA_ERR_ARG;
    if (m > VECCHIA_MAX_M) return VECCHIA_ERR_UNSUPPORTED;
    *log_p = NAN;
    *std_err = NAN;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    const bool dev = is_device_ptr(sites);
    if (is_device_ptr(u) != dev) return VECCHIA_ERR_ARG;
    const bool host_xy = order_kind == VECCHIA_ORDER_XY && D > vk::kOrderXyDeviceMax;
    Carve dv(nullptr);
    const size_t o_s = dv.off;
    if (!dev) dv.take<double>(2 * D);
    const size_t o_u = dv.off;
    if (!dev) dv.take<double>(D);
    const size_t o_perm = dv.off;
    dv.take<int32_t>(D);
    const size_t o_so = dv.off;
    dv.take<double>(2 * D);
    const size_t o_uo = dv.off;
    dv.take<double>(D);
    const size_t o_nbr = dv.off;
    dv.take<int32_t>((size_t)D * std::max(m, 1));
    const size_t o_bad = dv.off;
    dv.take<int>(1);
    const size_t o_scr = dv.off;
    dv.take<char>(std::max(std::max(vk::knn_scratch_bytes(D), vk::order_xy_scratch_bytes(D)),
                           order_kind == VECCHIA_ORDER_MAXMIN ? vk::maxmin_scratch_bytes(D) : (size_t)0));
    int st = ensure_aux(c, dv.off);
    if (st != VECCHIA_OK) return st;
    char* X = (char*)c->aux;
    const cudaStream_t s = c->stream;
    const double* sd = dev ? sites : (const double*)(X + o_s);
    const double* ud = dev ? u : (const double*)(X + o_u);
    int32_t* perm = (int32_t*)(X + o_perm);
    double* so = (double*)(X + o_so);
    double* uo = (double*)(X + o_uo);
    int32_t* nbr = (int32_t*)(X + o_nbr);
    cudaError_t e = cudaSuccess;
    if (!dev) {
        e = cudaMemcpyAsync(X + o_s, sites, sizeof(double) * 2 * D, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(X + o_u, u, sizeof(double) * D, cudaMemcpyHostToDevice, s);
    }
    // ordering, queued on the stream (the host sort only for XY beyond the device size)
    std::vector<int32_t> hp;
    if (e == cudaSuccess) {
        if (order_kind == VECCHIA_ORDER_MAXMIN) {
            e = vk::launch_maxmin(sd, D, perm, X + o_scr, s);
        } else if (order_kind == VECCHIA_ORDER_XY && !host_xy) {
            e = vk::launch_order_xy(sd, D, perm, X + o_scr, s);
        } else {
            hp.resize((size_t)D);
            if (order_kind == VECCHIA_ORDER_XY) {
                st = vecchia_order(dev ? c : nullptr, sites, D, VECCHIA_ORDER_XY, hp.data());
                if (st != VECCHIA_OK) return st;
            } else {
                for (int64_t k = 0; k < D; ++k) hp[(size_t)k] = (int32_t)k;
            }
            e = cudaMemcpyAsync(perm, hp.data(), sizeof(int32_t) * D, cudaMemcpyHostToDevice, s);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(X + o_bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = vk::launch_gather(perm, sd, ud, D, so, uo, (int*)(X + o_bad), s);
    if (e == cudaSuccess && m > 0) e = vk::launch_knn(so, D, m, nbr, X + o_scr, s);
    if (e == cudaSuccess && !hp.empty()) e = cudaStreamSynchronize(s);  // hp must outlive its upload
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    vecchia_problem p{};
    p.sites = so;
    p.nbr = m > 0 ? nbr : nullptr;
    p.u = uo;
    p.D = D;
    p.m = m;
    p.S = S;
    p.N = N;
    p.seed = seed;
    p.cov = cov;
    int32_t status = VECCHIA_OK;
    st = run_problems(c, &p, 1, precision, log_p, std_err, &status, nullptr, nullptr, nullptr);
    if (perm_out && (st == VECCHIA_OK || st == VECCHIA_ERR_NOT_PD)) {
        if (cudaMemcpyAsync(perm_out, perm, sizeof(int32_t) * D, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return VECCHIA_ERR_CUDA;
        }
    }
    return st;
}

int vecchia_neighbors(vecchia_ctx* c, const double* sites, int64_t D, int m, int32_t* nbr) {
    if (!c || !sites || D < 1 || D > INT_MAX / 2 || m < 0) return VECCHIA_ERR_ARG;
    if (m > VECCHIA_MAX_M) return VECCHIA_ERR_UNSUPPORTED;
    if (m == 0) return VECCHIA_OK;
    if (!nbr) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    const bool dev_in = is_device_ptr(sites), dev_out = is_device_ptr(nbr);
    Carve dv(nullptr);
    const size_t o_s = dv.off;
    if (!dev_in) dv.take<double>(2 * D);
    const size_t o_n = dv.off;
    if (!dev_out) dv.take<int32_t>((size_t)D * m);
    const size_t o_scr = dv.off;
    dv.take<char>(vk::knn_scratch_bytes(D));
    int st = ensure_arena(c, dv.off);
    if (st != VECCHIA_OK) return st;
    char* A = (char*)c->arena;
    const double* sd = dev_in ? sites : (const double*)(A + o_s);
    int32_t* nd = dev_out ? nbr : (int32_t*)(A + o_n);
    cudaError_t e = cudaSuccess;
    if (!dev_in) e = cudaMemcpyAsync(A + o_s, sites, sizeof(double) * 2 * D, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = vk::launch_knn(sd, D, m, nd, A + o_scr, c->stream);
    if (e == cudaSuccess && !dev_out)
        e = cudaMemcpyAsync(nbr, nd, sizeof(int32_t) * D * m, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return VECCHIA_OK;
}

int vecchia_neighbors_async(vecchia_ctx* c, const double* sites, int64_t D, int m, int32_t* nbr) {
    if (!c || !sites || D < 1 || D > INT_MAX / 2 || m < 0) return VECCHIA_ERR_ARG;
    if (m > VECCHIA_MAX_M) return VECCHIA_ERR_UNSUPPORTED;
    if (m == 0) return VECCHIA_OK;
    if (!nbr) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    int st = ensure_arena(c, vk::knn_scratch_bytes(D));
    if (st != VECCHIA_OK) return st;
    const cudaError_t e = vk::launch_knn(sites, D, m, nbr, c->arena, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return VECCHIA_OK;
}

int vecchia_log_cdf_terms(vecchia_ctx* c, const double* sites, int64_t D, const int32_t* nbr, int m,
                          vecchia_cov cov, const double* u, int64_t N, int S, uint64_t seed,
                          int precision, double* log_p, double* std_err, double* terms, double* num,
                          double* den) {
    vecchia_problem p{};
    p.sites = sites;
    p.nbr = nbr;
    p.u = u;
    p.D = D;
    p.m = m;
    p.S = S;
    p.N = N;
    p.seed = seed;
    p.cov = cov;
    int32_t status = VECCHIA_OK;
    double lp = NAN, se = NAN;
    const int st = run_problems(c, &p, 1, precision, &lp, &se, &status, terms, num, den);
    if (log_p) *log_p = lp;
    if (std_err) *std_err = se;
    return st;
}

int vecchia_log_cdf(vecchia_ctx* c, const double* sites, int64_t D, const int32_t* nbr, int m,
                    vecchia_cov cov, const double* u, int64_t N, int S, uint64_t seed, int precision,
                    double* log_p, double* std_err) {
    if (!log_p || !std_err) return VECCHIA_ERR_ARG;
    return vecchia_log_cdf_terms(c, sites, D, nbr, m, cov, u, N, S, seed, precision, log_p, std_err,
                                 nullptr, nullptr, nullptr);
}

int vecchia_grouped_log_cdf(vecchia_ctx* c, const double* sites, int64_t D, int p, const int32_t* cond,
                            int cmax, vecchia_cov cov, const double* u, int64_t N, int S, uint64_t seed,
                            int precision, double* log_p, double* std_err) {
    if (!log_p || !std_err || p < 1) return VECCHIA_ERR_ARG;
    vecchia_problem pr{};
    pr.sites = sites;
    pr.nbr = cond;
    pr.u = u;
    pr.D = D;
    pr.m = cmax;
    pr.S = S;
    pr.N = N;
    pr.seed = seed;
    pr.cov = cov;
    pr.group = p;
    // the largest conditioning set present picks the kernel instantiation
    // (rows are often much shorter than their width cmax)
    if (c && cond && cmax > 0 && D >= 1) {
        const int64_t G = (D + p - 1) / p;
        int cm = 0;
        if (is_device_ptr(cond)) {
            if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
            cudaError_t e = cudaSuccess;
            if (!c->small_dev) e = cudaMalloc(&c->small_dev, 256);
            if (e == cudaSuccess) e = vk::launch_rows_max(cond, G, cmax, c->small_dev, c->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&cm, c->small_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return VECCHIA_ERR_CUDA;
            }
        } else {
            for (int64_t k = 0; k < G; ++k) {
                const int32_t* row = cond + k * (int64_t)cmax;
                int n = 0;
                while (n < cmax && row[n] >= 0) ++n;
                cm = std::max(cm, n);
            }
        }
        pr.cond_max = cm;
    }
    int32_t status = VECCHIA_OK;
    return run_problems(c, &pr, 1, precision, log_p, std_err, &status, nullptr, nullptr, nullptr);
}

int vecchia_group_conditioning(vecchia_ctx* c, const double* sites, int64_t D, int p, int m, int method,
                               uint64_t seed, int cmax, int32_t* cond, int32_t* count) {
    if (!c || D < 1 || D > INT_MAX / 2 || p < 1 || m < 0 || cmax < 0) return VECCHIA_ERR_ARG;
    if (method != VECCHIA_COND_NEAREST && method != VECCHIA_COND_RANDOM) return VECCHIA_ERR_ARG;
    if (m > VECCHIA_MAX_M || cmax + p > VECCHIA_MAX_M + 1) return VECCHIA_ERR_UNSUPPORTED;
    if (method == VECCHIA_COND_RANDOM && m > cmax) return VECCHIA_ERR_ARG;
    if (method == VECCHIA_COND_NEAREST && !sites) return VECCHIA_ERR_ARG;
    const int64_t G = (D + p - 1) / p;
    if (cmax == 0) {
        if (count) {
            if (is_device_ptr(count)) {
                if (cudaSetDevice(c->device) != cudaSuccess ||
                    cudaMemsetAsync(count, 0, sizeof(int32_t) * G, c->stream) != cudaSuccess ||
                    cudaStreamSynchronize(c->stream) != cudaSuccess) {
                    cudaGetLastError();
                    return VECCHIA_ERR_CUDA;
                }
            } else {
                std::memset(count, 0, sizeof(int32_t) * G);
            }
        }
        return VECCHIA_OK;
    }
    if (!cond) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    const bool dev_out = is_device_ptr(cond);
    const bool dev_in = method == VECCHIA_COND_NEAREST && is_device_ptr(sites);
    if (count && is_device_ptr(count) != dev_out) return VECCHIA_ERR_ARG;
    const int mm = std::max(m, 1);
    Carve dv(nullptr);
    const size_t o_s = dv.off;
    if (method == VECCHIA_COND_NEAREST && !dev_in) dv.take<double>(2 * D);
    const size_t o_per = dv.off;
    if (method == VECCHIA_COND_NEAREST) dv.take<int32_t>((size_t)D * mm);
    const size_t o_cond = dv.off;
    if (!dev_out) dv.take<int32_t>((size_t)G * cmax);
    const size_t o_cnt = dv.off;
    dv.take<int32_t>((size_t)G);
    const size_t o_over = dv.off;
    dv.take<int>(1);
    const size_t o_scr = dv.off;
    if (method == VECCHIA_COND_NEAREST) dv.take<char>(vk::knn_scratch_bytes(D));
    int st = ensure_arena(c, dv.off);
    if (st != VECCHIA_OK) return st;
    char* A = (char*)c->arena;
    const cudaStream_t s = c->stream;
    int32_t* cd = dev_out ? cond : (int32_t*)(A + o_cond);
    int32_t* cnt = (count && dev_out) ? count : (int32_t*)(A + o_cnt);
    int* over = (int*)(A + o_over);
    cudaError_t e = cudaMemsetAsync(over, 0, sizeof(int), s);
    if (method == VECCHIA_COND_NEAREST) {
        const double* sd = dev_in ? sites : (const double*)(A + o_s);
        int32_t* per = (int32_t*)(A + o_per);
        if (e == cudaSuccess && !dev_in)
            e = cudaMemcpyAsync(A + o_s, sites, sizeof(double) * 2 * D, cudaMemcpyHostToDevice, s);
        if (m > 0) {
            if (e == cudaSuccess) e = vk::launch_knn(sd, D, m, per, A + o_scr, s, p);
        } else if (e == cudaSuccess) {
            e = cudaMemsetAsync(per, 0xff, sizeof(int32_t) * D, s);  // m = 0: one empty row per site
        }
        if (e == cudaSuccess) e = vk::launch_group_union(per, D, mm, p, cmax, cd, cnt, over, s);
    } else if (e == cudaSuccess) {
        e = vk::launch_group_random(D, p, m, seed, cmax, cd, cnt, s);
    }
    int h_over = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_over, over, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !dev_out)
        e = cudaMemcpyAsync(cond, cd, sizeof(int32_t) * G * cmax, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && count && !dev_out)
        e = cudaMemcpyAsync(count, cnt, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return h_over ? VECCHIA_ERR_ARG : VECCHIA_OK;
}

int vecchia_full_genz(vecchia_ctx* c, const double* sites, int64_t D, vecchia_cov cov, const double* u, int64_t N,
                      int S, uint64_t seed, int precision, double* log_p, double* rel_se) {
    if (!c || !sites || !u || !log_p || !rel_se || D < 1 || N < 1 || N > INT_MAX) return VECCHIA_ERR_ARG;
    if (S < 2 || S > VECCHIA_MAX_S || !cov_ok(cov)) return VECCHIA_ERR_ARG;
    if (precision != VECCHIA_FP64 && precision != VECCHIA_MIXED) return VECCHIA_ERR_ARG;
    if (D > VECCHIA_FULL_MAX_D) return VECCHIA_ERR_UNSUPPORTED;
    *log_p = NAN;
    *rel_se = NAN;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    c->last_error_site = -1;
    const bool mixed = precision == VECCHIA_MIXED;
    const bool dev_in = is_device_ptr(sites);
    if (dev_in != is_device_ptr(u)) return VECCHIA_ERR_ARG;
    const int64_t dim = D > 1 ? D - 1 : 1;
    std::vector<uint32_t> g((size_t)dim), gfix((size_t)dim);
    lattice_host(N, (int)dim, g.data());
    for (int64_t j = 0; j < dim; ++j)  // round(g 2^32 / N)
        gfix[(size_t)j] = (uint32_t)((((uint64_t)g[(size_t)j] << 32) + (uint64_t)N / 2) / (uint64_t)N);
    Carve dv(nullptr);
    const size_t o_s = dv.off;
    if (!dev_in) dv.take<double>(2 * D);
    const size_t o_u = dv.off;
    if (!dev_in) dv.take<double>(D);
    const size_t o_scr = dv.off;
    dv.take<char>(vk::full_genz_scratch_bytes(D, N, S, mixed));
    int st = ensure_arena(c, dv.off);
    if (st != VECCHIA_OK) return st;
    char* A = (char*)c->arena;
    const double* sd = dev_in ? sites : (const double*)(A + o_s);
    const double* ud = dev_in ? u : (const double*)(A + o_u);
    const int64_t bps = vk::full_genz_blocks_per_shift(N, mixed);
    std::vector<double> part((size_t)(S * bps));
    int bad = INT_MAX, timed_out = 0;
    cudaError_t e = cudaSuccess;
    if (!dev_in) e = cudaMemcpyAsync(A + o_s, sites, sizeof(double) * 2 * D, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !dev_in)
        e = cudaMemcpyAsync(A + o_u, u, sizeof(double) * D, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = vk::launch_full_genz(sd, ud, D, cov, N, S, mixed, g.data(), gfix.data(), seed, A + o_scr, part.data(),
                                 &bad, &timed_out, c->full_wait_ns, c->full_withhold,
                                 c->timing ? c->ev0 : nullptr, c->timing ? c->ev1 : nullptr, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    if (c->timing) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->genz_ms = ms;
    }
    if (bad != INT_MAX) {
        c->last_error_site = bad;
        return VECCHIA_ERR_NOT_PD;
    }
    if (timed_out) return VECCHIA_ERR_TIMEOUT;
    // per-shift means (tile sums in order), their mean and relative standard error
    std::vector<double> ps((size_t)S);
    double mean = 0.0;
    for (int s = 0; s < S; ++s) {
        double t = 0.0;
        for (int64_t b = 0; b < bps; ++b) t += part[(size_t)(s * bps + b)];
        ps[(size_t)s] = t / (double)N;
        mean += ps[(size_t)s];
    }
    mean /= (double)S;
    double ss = 0.0;
    for (int s = 0; s < S; ++s) ss += (ps[(size_t)s] - mean) * (ps[(size_t)s] - mean);
    *log_p = std::log(mean);
    *rel_se = std::sqrt(ss / ((double)S * (S - 1))) / mean;
    if (!std::isfinite(*log_p) || !std::isfinite(*rel_se)) return VECCHIA_ERR_NONFINITE;
    return VECCHIA_OK;
}

int vecchia_full_cholesky(vecchia_ctx* c, const double* sites, int64_t D, vecchia_cov cov, int precision,
                          double* L) {
    if (!c || !sites || !L || D < 1 || !cov_ok(cov)) return VECCHIA_ERR_ARG;
    if (precision != VECCHIA_FP64 && precision != VECCHIA_MIXED) return VECCHIA_ERR_ARG;
    if (D > VECCHIA_FULL_MAX_D) return VECCHIA_ERR_UNSUPPORTED;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    c->last_error_site = -1;
    const bool mixed = precision == VECCHIA_MIXED;
    const bool dev_in = is_device_ptr(sites), dev_out = is_device_ptr(L);
    Carve dv(nullptr);
    const size_t o_s = dv.off;
    if (!dev_in) dv.take<double>(2 * D);
    const size_t o_a = dv.off;
    dv.take<double>((size_t)D * D);
    const size_t o_t = dv.off;
    if (mixed) dv.take<char>(vk::chol_tc_scratch_bytes(D));
    const size_t o_b = dv.off;
    dv.take<int>(2);
    int st = ensure_arena(c, dv.off);
    if (st != VECCHIA_OK) return st;
    char* X = (char*)c->arena;
    const double* sd = dev_in ? sites : (const double*)(X + o_s);
    double* Ad = (double*)(X + o_a);
    int* bd = (int*)(X + o_b);
    const int status_init[2] = {INT_MAX, 0};
    int status[2] = {INT_MAX, 0};
    cudaError_t e = cudaSuccess;
    if (!dev_in) e = cudaMemcpyAsync(X + o_s, sites, sizeof(double) * 2 * D, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(Ad, 0, sizeof(double) * (size_t)D * D, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bd, status_init, sizeof(status_init), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = mixed ? vk::launch_cov_chol(sd, D, cov, Ad, bd, c->stream, X + o_t, bd + 1, c->full_wait_ns)
                  : vk::launch_cov_chol(sd, D, cov, Ad, bd, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L, Ad, sizeof(double) * (size_t)D * D,
                            dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status, bd, sizeof(status), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    if (status[0] != INT_MAX) {
        c->last_error_site = status[0];
        return VECCHIA_ERR_NOT_PD;
    }
    return status[1] ? VECCHIA_ERR_TIMEOUT : VECCHIA_OK;
}

int vecchia_mixture_log_cdf(vecchia_ctx* c, const double* sites, int64_t D, const int32_t* nbr, int m,
                            vecchia_cov cov, const double* x, int64_t N, int S, uint64_t seed,
                            double beta, double gamma, int n_nodes, int precision, double* log_g,
                            double* std_err) {
    if (!c || !log_g || !std_err) return VECCHIA_ERR_ARG;
    if (!(beta >= 0.0) || !(gamma > 0.0) || !std::isfinite(beta) || !std::isfinite(gamma) || n_nodes < 1 ||
        n_nodes > 256)
        return VECCHIA_ERR_ARG;
    *log_g = NAN;
    *std_err = NAN;
    std::vector<double> rq, w;
    mixture_nodes(n_nodes, beta, gamma, rq, w);
    std::vector<vecchia_problem> probs(n_nodes);
    for (int q = 0; q < n_nodes; ++q) {
        const double r = rq[q];
        vecchia_problem& p = probs[q];
        p.sites = sites;
        p.nbr = nbr;
        p.u = x;
        p.D = D;
        p.m = m;
        p.S = S;
        p.N = N;
        p.seed = seed;
        p.cov = cov;
        p.cov.variance = cov.variance * r * r;  // Phi_D(x / r; Sigma) = Phi_D(x; r^2 Sigma)
        p.cov.nugget = cov.nugget * r * r;
    }
    std::vector<double> lp(n_nodes), se(n_nodes);
    std::vector<int32_t> st(n_nodes);
    int rc = run_problems(c, probs.data(), n_nodes, precision, lp.data(), se.data(), st.data(), nullptr,
                          nullptr, nullptr);
    if (rc != VECCHIA_OK) return rc;
    for (int q = 0; q < n_nodes; ++q)
        if (st[q] != VECCHIA_OK) return st[q];
    // log G = log sum_q w_q P_q, in a fixed order with the largest term factored out
    double mx = -INFINITY;
    for (int q = 0; q < n_nodes; ++q) mx = std::max(mx, std::log(w[q]) + lp[q]);
    double sum = 0.0;
    for (int q = 0; q < n_nodes; ++q) sum += std::exp(std::log(w[q]) + lp[q] - mx);
    *log_g = mx + std::log(sum);
    // the nodes share shifts (correlated errors): bound by full correlation
    double seb = 0.0;
    for (int q = 0; q < n_nodes; ++q) seb += std::exp(std::log(w[q]) + lp[q] - *log_g) * se[q];
    *std_err = seb;
    return VECCHIA_OK;
}

int vecchia_censored_log_cdf(vecchia_ctx* c, const double* sites_c, int64_t nc, const int32_t* nbr, int m,
                             const double* sites_i, int64_t ni, vecchia_cov cov, const double* x_c,
                             const double* x_i, int64_t N, int S, uint64_t seed, double beta, double gamma,
                             int n_nodes, int precision, double* log_g, double* std_err) {
    if (!c || !log_g || !std_err || nc < 0 || ni < 0 || nc + ni < 1) return VECCHIA_ERR_ARG;
    if ((nc > 0 && (!sites_c || !x_c || (m > 0 && !nbr))) || (ni > 0 && (!sites_i || !x_i))) return VECCHIA_ERR_ARG;
    if (n_nodes < 0 || n_nodes > 256 || m < 0) return VECCHIA_ERR_ARG;
    if (n_nodes > 0 && (!(beta >= 0.0) || !(gamma > 0.0) || !std::isfinite(beta) || !std::isfinite(gamma)))
        return VECCHIA_ERR_ARG;
    if (!cov_ok(cov) || S < 2 || S > VECCHIA_MAX_S || N < 1 || N > INT_MAX) return VECCHIA_ERR_ARG;
    if (precision != VECCHIA_FP64 && precision != VECCHIA_MIXED) return VECCHIA_ERR_ARG;
    if (ni > VECCHIA_CENSOR_MAX_OBS || nc > INT_MAX / 2 || m > VECCHIA_MAX_M) return VECCHIA_ERR_UNSUPPORTED;
    *log_g = NAN;
    *std_err = NAN;
    if (ni == 0)  // nothing observed: the CDF itself (Eq. model03, or Phi_D when R = 1)
        return n_nodes == 0 ? vecchia_log_cdf(c, sites_c, nc, nbr, m, cov, x_c, N, S, seed, precision, log_g, std_err)
                            : vecchia_mixture_log_cdf(c, sites_c, nc, nbr, m, cov, x_c, N, S, seed, beta, gamma,
                                                      n_nodes, precision, log_g, std_err);
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    c->last_error_site = -1;
    const bool dev = is_device_ptr(sites_i);
    if (is_device_ptr(x_i) != dev || (nc > 0 && (is_device_ptr(sites_c) != dev || is_device_ptr(x_c) != dev)) ||
        (nc > 0 && m > 0 && is_device_ptr(nbr) != dev))
        return VECCHIA_ERR_ARG;
    const int k = (int)ni;
    Carve dv(nullptr);
    const size_t o_si = dv.off;
    if (!dev) dv.take<double>(2 * ni);
    const size_t o_xi = dv.off;
    if (!dev) dv.take<double>(ni);
    const size_t o_sc = dv.off;
    if (!dev) dv.take<double>(2 * nc);
    const size_t o_xc = dv.off;
    if (!dev) dv.take<double>(nc);
    const size_t o_nb = dv.off;
    if (!dev && m > 0) dv.take<int32_t>((size_t)nc * m);
    const size_t o_L = dv.off;
    dv.take<double>((size_t)k * k);
    const size_t o_V = dv.off;
    dv.take<double>((size_t)(nc + 1) * k);
    const size_t o_u = dv.off;
    dv.take<double>(nc);
    const size_t o_bad = dv.off;
    dv.take<int>(1);
    int st = ensure_aux(c, dv.off);
    if (st != VECCHIA_OK) return st;
    char* X = (char*)c->aux;
    const cudaStream_t s = c->stream;
    const double* si = dev ? sites_i : (const double*)(X + o_si);
    const double* xi = dev ? x_i : (const double*)(X + o_xi);
    const double* sc = dev ? sites_c : (const double*)(X + o_sc);
    const double* xc = dev ? x_c : (const double*)(X + o_xc);
    const int32_t* nb = (dev || m == 0) ? nbr : (const int32_t*)(X + o_nb);
    double* L = (double*)(X + o_L);
    double* V = (double*)(X + o_V);
    double* ud = (double*)(X + o_u);
    int* bad = (int*)(X + o_bad);
    cudaError_t e = cudaSuccess;
    if (!dev) {
        e = cudaMemcpyAsync(X + o_si, sites_i, sizeof(double) * 2 * ni, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(X + o_xi, x_i, sizeof(double) * ni, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && nc > 0)
            e = cudaMemcpyAsync(X + o_sc, sites_c, sizeof(double) * 2 * nc, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && nc > 0) e = cudaMemcpyAsync(X + o_xc, x_c, sizeof(double) * nc, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && nc > 0 && m > 0)
            e = cudaMemcpyAsync(X + o_nb, nbr, sizeof(int32_t) * nc * m, cudaMemcpyHostToDevice, s);
    }
    const int badinit = INT_MAX;
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad, &badinit, sizeof(int), cudaMemcpyHostToDevice, s);
    // Sigma_II = L L^T; V = L^-1 Sigma_Ic, w = L^-1 x_I, thresholds x_c - V w
    if (e == cudaSuccess) e = vk::launch_cov_chol(si, ni, cov, L, bad, s);
    if (e == cudaSuccess) e = vk::launch_conditioning(L, k, si, xi, sc, xc, nc, cov, V, ud, s);
    std::vector<double> diag((size_t)k), w((size_t)k);
    int hbad = INT_MAX;
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(diag.data(), sizeof(double), L, sizeof(double) * (k + 1), sizeof(double), k,
                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.data(), V + (size_t)nc * k, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    if (hbad != INT_MAX) {
        c->last_error_site = hbad;  // index among the observed sites
        return VECCHIA_ERR_NOT_PD;
    }
    // log phi_k(x_I / r; Sigma_II) - k log r = -k/2 log 2 pi - log det L - |w|^2 / (2 r^2) - k log r
    double logdetL = 0.0, quad = 0.0;
    for (int t = 0; t < k; ++t) {
        logdetL += std::log(diag[(size_t)t]);
        quad += w[(size_t)t] * w[(size_t)t];
    }
    const double kLog2Pi = 1.8378770664093454836;
    auto log_dens = [&](double r) { return -0.5 * k * kLog2Pi - logdetL - quad / (2.0 * r * r) - k * std::log(r); };
    std::vector<double> rq, wq;
    if (n_nodes == 0) {
        rq.assign(1, 1.0);
        wq.assign(1, 1.0);
    } else {
        mixture_nodes(n_nodes, beta, gamma, rq, wq);
    }
    const int nq = (int)rq.size();
    std::vector<double> lp((size_t)nq, 0.0), se((size_t)nq, 0.0);
    if (nc > 0) {
        std::vector<vecchia_problem> probs((size_t)nq);
        std::vector<double> scale((size_t)nq);
        for (int q = 0; q < nq; ++q) {
            vecchia_problem& p = probs[(size_t)q];
            const double r2 = rq[(size_t)q] * rq[(size_t)q];
            p.sites = sc;
            p.nbr = nb;
            p.u = ud;
            p.D = nc;
            p.m = m;
            p.S = S;
            p.N = N;
            p.seed = seed;
            p.cov = cov;  // Phi_c(y / r; Sigma_{c|I}) = Phi_c(y; r^2 Sigma_{c|I})
            p.cov.variance = cov.variance * r2;
            p.cov.nugget = cov.nugget * r2;
            scale[(size_t)q] = r2;
        }
        std::vector<int32_t> stv((size_t)nq);
        int rc = run_problems(c, probs.data(), nq, precision, lp.data(), se.data(), stv.data(), nullptr, nullptr,
                              nullptr, V, k, scale.data());
        if (rc != VECCHIA_OK) return rc;
        for (int q = 0; q < nq; ++q)
            if (stv[(size_t)q] != VECCHIA_OK) return stv[(size_t)q];
    }
    // log G_I = log sum_q w_q exp(lp_q + log density(r_q)), largest term factored out
    std::vector<double> tq((size_t)nq);
    double mx = -INFINITY;
    for (int q = 0; q < nq; ++q) {
        tq[(size_t)q] = std::log(wq[(size_t)q]) + lp[(size_t)q] + log_dens(rq[(size_t)q]);
        mx = std::max(mx, tq[(size_t)q]);
    }
    double sum = 0.0;
    for (int q = 0; q < nq; ++q) sum += std::exp(tq[(size_t)q] - mx);
    *log_g = mx + std::log(sum);
    double seb = 0.0;  // the nodes share shifts: bound by full correlation
    for (int q = 0; q < nq; ++q) seb += std::exp(tq[(size_t)q] - *log_g) * se[(size_t)q];
    *std_err = seb;
    if (!std::isfinite(*log_g)) return VECCHIA_ERR_NONFINITE;
    return VECCHIA_OK;
}

int vecchia_log_cdf_batch(vecchia_ctx* c, const vecchia_problem* probs, int n_probs, int precision,
                          double* log_p, double* std_err, int32_t* status) {
    if (!c || !probs || n_probs < 1 || !log_p || !std_err || !status) return VECCHIA_ERR_ARG;
    return run_problems(c, probs, n_probs, precision, log_p, std_err, status, nullptr, nullptr, nullptr);
}

int vecchia_result_init(vecchia_ctx* c, vecchia_result* results, int n) {
    if (!c || n < 0 || (n > 0 && !results)) return VECCHIA_ERR_ARG;
    if (n == 0) return VECCHIA_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    const cudaError_t e = vk::launch_init_results((ProbResult*)results, n, nullptr, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return VECCHIA_OK;
}

int vecchia_partials_async(vecchia_ctx* c, const vecchia_segment* segs, int n, int precision) {
    if (!c || n < 0 || (n > 0 && !segs)) return VECCHIA_ERR_ARG;
    if (precision != VECCHIA_FP64 && precision != VECCHIA_MIXED) return VECCHIA_ERR_ARG;
    if (n == 0) return VECCHIA_OK;
    for (int i = 0; i < n; ++i)
        if (!segment_ok(segs[i])) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    const bool mixed = precision == VECCHIA_MIXED;
    int64_t bucket_sites[NB] = {0}, total_sites = 0, shift_rows = 0;
    int bucket_segs[NB] = {0}, max_S[NB] = {0}, max_S_all = 0, max_bucket = 0;
    std::vector<int> bk(n);
    std::vector<uint32_t*> lat(n);
    for (int i = 0; i < n; ++i) {
        const auto& p = segs[i].prob;
        bk[i] = vk::bucket_of(vk::max_term_dim(p.m, p.group, p.cond_max));
        max_S_all = std::max(max_S_all, p.S);
        max_bucket = std::max(max_bucket, bk[i]);
        shift_rows += p.S;
        bucket_sites[bk[i]] += segs[i].site_count;
        bucket_segs[bk[i]] += segs[i].site_count > 0;
        max_S[bk[i]] = std::max(max_S[bk[i]], p.S);
        total_sites += segs[i].site_count;
        lat[i] = lattice_for(c, p.N);
        if (!lat[i]) return VECCHIA_ERR_NOMEM;
    }
    GenzTile tiles[NB];
    int max_groups = 1;
    for (int b = 0; b < NB; ++b) {
        tiles[b] = c->tile_set[mixed][b] ? c->tile[mixed][b]
                                         : default_tile(mixed, total_sites, std::max(max_S[b], 2), b);
        max_groups = std::max(max_groups, tiles[b].groups);
    }
    const int64_t fb_cap =
        mixed ? std::max<int64_t>(total_sites * max_groups + vk::genz_items_slack(vk::device_sm_count(c->device)), 1)
              : 1;
    Carve dv(nullptr);
    const size_t o_delta = dv.off;
    dv.take<double>((size_t)shift_rows * kDim);
    const size_t o_dfix = dv.off;
    dv.take<uint32_t>((size_t)shift_rows * kDim);
    const size_t o_fbc = dv.off;
    dv.take<int>(1);
    const size_t o_fbi = dv.off;
    dv.take<int2>((size_t)fb_cap);
    Carve hb(nullptr);
    const size_t b_probs = hb.off;
    hb.take<ProbDev>(n);
    const size_t b_seeds = hb.off;
    hb.take<uint64_t>(n);
    const size_t b_S = hb.off;
    hb.take<int32_t>(n);
    const size_t b_off = hb.off;
    hb.take<int64_t>(n);
    size_t b_segp[NB], b_segb[NB];
    for (int b = 0; b < NB; ++b) {
        b_segp[b] = hb.off;
        hb.take<int>(bucket_segs[b] + 1);
        b_segb[b] = hb.off;
        hb.take<int2>(std::max(bucket_segs[b], 1));
    }
    const size_t blob_bytes = hb.off;
    const size_t o_blob = dv.off;
    dv.take<char>(blob_bytes);
    int st = ensure_arena(c, dv.off);
    if (st != VECCHIA_OK) return st;
    int which = 0;
    char* H = async_stage(c, blob_bytes, &which);
    if (!H) return VECCHIA_ERR_NOMEM;
    char* A = (char*)c->arena;
    ProbDev* hp = (ProbDev*)(H + b_probs);
    for (int i = 0, off = 0; i < n; off += segs[i].prob.S * kDim, ++i) {
        fill_probdev(hp[i], segs[i], lat[i], A, o_delta, o_dfix, off);
        ((uint64_t*)(H + b_seeds))[i] = segs[i].prob.seed;
        ((int32_t*)(H + b_S))[i] = segs[i].prob.S;
        ((int64_t*)(H + b_off))[i] = off;
    }
    for (int b = 0; b < NB; ++b) {
        int* sp = (int*)(H + b_segp[b]);
        int2* sb = (int2*)(H + b_segb[b]);
        int k = 0, run = 0;
        for (int i = 0; i < n; ++i) {
            if (bk[i] != b || segs[i].site_count <= 0) continue;
            sp[k] = run;
            sb[k] = make_int2(i, (int)segs[i].site_begin);
            run += (int)segs[i].site_count;
            ++k;
        }
        sp[k] = run;
    }
    const cudaStream_t s = c->stream;
    char* blob = A + o_blob;
    int* fbc = (int*)(A + o_fbc);
    cudaError_t e = cudaMemcpyAsync(blob, H, blob_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->astage_ev[which], s);
    if (e == cudaSuccess) e = vk::launch_init_results(nullptr, 0, fbc, s);
    if (e == cudaSuccess)
        e = vk::launch_shifts((const uint64_t*)(blob + b_seeds), (const int32_t*)(blob + b_S),
                              (const int64_t*)(blob + b_off), n, kDim, (double*)(A + o_delta),
                              (uint32_t*)(A + o_dfix), s);
    ProbDev* probs_d = (ProbDev*)(blob + b_probs);
    for (int b = NB - 1; b >= 0 && e == cudaSuccess; --b) {
        if (!bucket_sites[b]) continue;
        e = vk::launch_genz(b, mixed, tiles[b], probs_d, (const int*)(blob + b_segp[b]),
                            (const int2*)(blob + b_segb[b]), bucket_segs[b], (int)bucket_sites[b], nullptr,
                            fbc, (int2*)(A + o_fbi), max_S[b], (int)fb_cap, s);
    }
    if (mixed && e == cudaSuccess)
        e = vk::launch_genz_fallback(max_bucket, probs_d, fbc, (int2*)(A + o_fbi), (int)fb_cap, nullptr, max_S_all, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return VECCHIA_OK;
}

int vecchia_reduce_async(vecchia_ctx* c, const vecchia_segment* probs, int n) {
    if (!c || n < 0 || (n > 0 && !probs)) return VECCHIA_ERR_ARG;
    if (n == 0) return VECCHIA_OK;
    for (int i = 0; i < n; ++i)
        if (!segment_ok(probs[i])) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    int64_t scratch = 0, max_slices = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t T = vk::n_terms_of(probs[i].prob.D, probs[i].prob.group);
        scratch += vk::logsum_scratch(T, probs[i].prob.S);
        max_slices = std::max(max_slices, vk::logsum_slices(T));
    }
    Carve dv(nullptr);
    const size_t o_scr = dv.off;
    dv.take<double>(scratch);
    Carve hb(nullptr);
    const size_t b_probs = hb.off;
    hb.take<ProbDev>(n);
    const size_t b_off = hb.off;
    hb.take<int64_t>(n);
    const size_t blob_bytes = hb.off;
    const size_t o_blob = dv.off;
    dv.take<char>(blob_bytes);
    int st = ensure_arena(c, dv.off);
    if (st != VECCHIA_OK) return st;
    int which = 0;
    char* H = async_stage(c, blob_bytes, &which);
    if (!H) return VECCHIA_ERR_NOMEM;
    char* A = (char*)c->arena;
    int64_t run = 0;
    for (int i = 0; i < n; ++i) {
        fill_probdev(((ProbDev*)(H + b_probs))[i], probs[i], nullptr, A, 0, 0, 0);
        ((int64_t*)(H + b_off))[i] = run;
        run += vk::logsum_scratch(vk::n_terms_of(probs[i].prob.D, probs[i].prob.group), probs[i].prob.S);
    }
    const cudaStream_t s = c->stream;
    char* blob = A + o_blob;
    cudaError_t e = cudaMemcpyAsync(blob, H, blob_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->astage_ev[which], s);
    if (e == cudaSuccess)
        e = vk::launch_logsum((const ProbDev*)(blob + b_probs), n, (int)max_slices, nullptr, nullptr,
                              (double*)(A + o_scr), (const int64_t*)(blob + b_off), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return VECCHIA_OK;
}

int vecchia_plan_create(vecchia_ctx* c, const vecchia_problem* probs, int n_probs, int precision,
                        vecchia_plan** out, int32_t* status) {
    if (!c || !probs || n_probs < 1 || !out || !status) return VECCHIA_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    vecchia_plan* P = new (std::nothrow) vecchia_plan();
    if (!P) return VECCHIA_ERR_NOMEM;
    P->c = c;
    int st = prepare(c, probs, n_probs, precision, status, false, false, P->B);
    if (st != VECCHIA_OK) {
        plan_free(P);
        return st;
    }
    cudaError_t e = cudaMalloc((void**)&P->A, P->B.arena_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&P->H, P->B.blob_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan_free(P);
        return VECCHIA_ERR_NOMEM;
    }
    fill_blob(P->B, P->A, P->H, nullptr);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ready, cudaEventDisableTiming);
    // inputs become resident: host arrays are copied once, device arrays are read in place
    if (e == cudaSuccess) e = cudaEventRecord(P->ready, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ready, 0);
    if (e == cudaSuccess) e = stage_inputs(P->B, P->A, P->stream);
    // one eager run (also warms host-side launch caches), then capture the sequence
    if (e == cudaSuccess) e = enqueue(P->B, P->A, P->H, P->stream, false, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = enqueue(P->B, P->A, P->H, P->stream, false, nullptr);
        e = cudaStreamEndCapture(P->stream, &P->graph);
        if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan_free(P);
        return VECCHIA_ERR_CUDA;
    }
    *out = P;
    return VECCHIA_OK;
}

int vecchia_plan_run(vecchia_plan* P, const uint64_t* seeds, const vecchia_cov* covs, double* log_p,
                     double* std_err, int32_t* status) {
    if (!P || !log_p || !std_err || !status) return VECCHIA_ERR_ARG;
    const Batch& B = P->B;
    if (covs)
        for (int i = 0; i < B.n; ++i)
            if (B.ok[i] && !cov_ok(covs[i])) return VECCHIA_ERR_ARG;
    if (cudaSetDevice(P->c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    ProbDev* hp = (ProbDev*)(P->H + B.b_probs);
    uint64_t* hseeds = (uint64_t*)(P->H + B.b_seeds);
    for (int i = 0; i < B.n; ++i) {
        if (seeds) hseeds[i] = seeds[i];
        if (covs && B.ok[i]) set_cov(hp[i], covs[i]);
        status[i] = B.ok[i] ? VECCHIA_OK : VECCHIA_ERR_ARG;
    }
    cudaError_t e = cudaEventRecord(P->ready, P->c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ready, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(P->exec, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    P->c->last_error_site = -1;
    collect(B, P->H, log_p, std_err, status, &P->c->last_error_site);
    return VECCHIA_OK;
}

int vecchia_plan_destroy(vecchia_plan* P) {
    if (!P) return VECCHIA_ERR_ARG;
    cudaSetDevice(P->c->device);
    plan_free(P);
    return VECCHIA_OK;
}

int vecchia_set_tile(vecchia_ctx* c, int precision, int bucket, int warps, int points, int slices,
                     int groups) {
    if (!c || (precision != VECCHIA_FP64 && precision != VECCHIA_MIXED) || bucket < -1 ||
        bucket >= vk::kNumBuckets)
        return VECCHIA_ERR_ARG;
    if (warps < 1 || warps > 16 || (points != 1 && points != 2) || slices < 1 ||
        groups < 1 || groups > VECCHIA_MAX_S)
        return VECCHIA_ERR_ARG;
    const int b0 = bucket < 0 ? 0 : bucket, b1 = bucket < 0 ? vk::kNumBuckets - 1 : bucket;
    for (int b = b0; b <= b1; ++b) {
        c->tile[precision][b] = vk::GenzTile{warps, precision == VECCHIA_FP64 ? 1 : points, slices, groups};
        c->tile_set[precision][b] = true;
    }
    return VECCHIA_OK;
}

int vecchia_reset_tiles(vecchia_ctx* c) {
    if (!c) return VECCHIA_ERR_ARG;
    for (int p = 0; p < 2; ++p)
        for (int b = 0; b < vk::kNumBuckets; ++b) c->tile_set[p][b] = false;
    return VECCHIA_OK;
}

int vecchia_eval_special(vecchia_ctx* c, int which, const float* x, int64_t n, float* out) {
    if (!c || which < 0 || which > 7 || n < 0 || (n > 0 && (!x || !out))) return VECCHIA_ERR_ARG;
    if (n == 0) return VECCHIA_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    if (!is_device_ptr(x) || !is_device_ptr(out)) return VECCHIA_ERR_ARG;
    cudaError_t e = vk::launch_eval_special(which, x, n, out, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return VECCHIA_OK;
}

int vecchia_eval_special64(vecchia_ctx* c, int which, const double* x, int64_t n, double* out) {
    if (!c || which < 0 || which > 3 || n < 0 || (n > 0 && (!x || !out))) return VECCHIA_ERR_ARG;
    if (n == 0) return VECCHIA_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return VECCHIA_ERR_CUDA;
    if (!is_device_ptr(x) || !is_device_ptr(out)) return VECCHIA_ERR_ARG;
    cudaError_t e = vk::launch_eval_special64(which, x, n, out, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    return VECCHIA_OK;
}

int vecchia_set_timing(vecchia_ctx* c, int enable) {
    if (!c) return VECCHIA_ERR_ARG;
    c->timing = enable != 0;
    return VECCHIA_OK;
}

int vecchia_genz_time_ms(const vecchia_ctx* c, double* ms) {
    if (!c || !ms) return VECCHIA_ERR_ARG;
    *ms = c->genz_ms;
    return VECCHIA_OK;
}

int vecchia_set_full_genz_wait(vecchia_ctx* c, uint64_t limit_ns, int withhold) {
    if (!c) return VECCHIA_ERR_ARG;
    c->full_wait_ns = limit_ns;
    c->full_withhold = withhold ? 1 : 0;
    return VECCHIA_OK;
}

}  // extern "C"
