// noalloc.cu -- vecchia_log_cdf_noalloc: the log-CDF without any allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// log-CDF: programs whose allocator owns the whole device and forbids foreign
// cudaMalloc calls, code that must run within a fixed memory budget (no
// allocation after start-up), or hosts that have no context object of ours.  This entry point runs the same
// kernels as vecchia_log_cdf but keeps every piece of scratch (per-shift
// partial sums, shift tables, lattice table, parameters, results) in one
// file-scope device array of fixed size, so it calls no cudaMalloc, no
// cudaFree, no cudaMallocHost and no other allocating routine.
//
// The array is part of the library's device image: every GPU that loads the
// library holds VECCHIA_NOALLOC_SCRATCH_BYTES of it until the process exits.
// All calls share it and it keeps the last call's contents, so the pieces
// that must start at zero are cleared on the stream by every call, and calls
// whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on it: callers must serialise them.
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "vk_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[VECCHIA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of g_scratch on `device` (which must be current).  Looked up
// once per device; the name g_scratch in host code is only a stand-in.
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return VECCHIA_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return VECCHIA_ERR_CUDA;
        }
        g_scratch_dev[device] = p;
    }
    *out = (unsigned char*)g_scratch_dev[device];
    return VECCHIA_OK;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// True if p is device (or managed) memory that lives on `device`.
bool device_array(const void* p, int device) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

// Makes `device` current for the call and puts the caller's device back on
// every return path.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        ok = cudaSetDevice(device) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool cov_valid(const vecchia_cov& c) {
    if (!(c.variance > 0.0) || !(c.range > 0.0) || !(c.nugget >= 0.0)) return false;
    if (!std::isfinite(c.variance) || !std::isfinite(c.range) || !std::isfinite(c.nugget)) return false;
    if (c.kind == VECCHIA_COV_EXPONENTIAL) return true;
    if (c.kind == VECCHIA_COV_MATERN) return c.nu == 0.5 || c.nu == 1.5 || c.nu == 2.5;
    if (c.kind == VECCHIA_COV_ANISO_EXP)
        return std::isfinite(c.angle) && std::isfinite(c.aspect) && c.aspect > 0.0;
    return false;
}

}  // namespace

extern "C" int vecchia_log_cdf_noalloc(int device, void* cuda_stream, const double* sites_ordered,
                                       int64_t D, const int32_t* nbr, int m, vecchia_cov cov,
                                       const double* u, int64_t N, int S, uint64_t seed,
                                       int precision, double* log_p, double* std_err) {
    using vk::ProbDev;
    using vk::ProbResult;
    if (!log_p || !std_err || !sites_ordered || !u || D < 1 || D > INT_MAX / 2) return VECCHIA_ERR_ARG;
    if (m < 0 || (m > 0 && !nbr)) return VECCHIA_ERR_ARG;
    if (m > VECCHIA_MAX_M) return VECCHIA_ERR_UNSUPPORTED;
    if (N < 1 || N > INT_MAX || S < 2 || S > VECCHIA_MAX_S || !cov_valid(cov)) return VECCHIA_ERR_ARG;
    if (precision != VECCHIA_FP64 && precision != VECCHIA_MIXED) return VECCHIA_ERR_ARG;
    *log_p = NAN;
    *std_err = NAN;
    const DeviceGuard guard(device);
    if (!guard.ok) return VECCHIA_ERR_ARG;
    if (!device_array(sites_ordered, device) || !device_array(u, device) ||
        (m > 0 && !device_array(nbr, device)))
        return VECCHIA_ERR_ARG;
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool mixed = precision == VECCHIA_MIXED;
    constexpr int kDim = vk::kMaxDim;

    // tile: the built-in rule of vecchia_log_cdf (mixed: two points per lane up
    // to 32 variables, 8 warps above 21; power-of-two shift groups for ~2048
    // CTA items (4096 up to 16 variables), never fewer shifts per item than
    // warps; above 32 variables 8
    // warps, one point, one group)
    const int bucket = vk::bucket_of(m + 1);
    const int dmax = vk::kDmaxBuckets[bucket];
    const int warps = (mixed && dmax > 21) ? 8 : 4;
    int groups = 1;
    const int64_t target = dmax <= 16 ? 4096 : 2048;
    while (groups < S && (int64_t)groups * D < target && S / (2 * groups) >= warps) groups *= 2;
    vk::GenzTile tile{warps, mixed ? 2 : 1, 1, groups};
    if (dmax > 32) tile = vk::GenzTile{8, 1, 1, 1};

    // scratch layout (every offset a multiple of 256 bytes)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += up256(bytes > 0 ? bytes : 1);
        return o;
    };
    const size_t o_num = take(sizeof(double) * (size_t)D * S);
    const size_t o_den = take(sizeof(double) * (size_t)D * S);
    const size_t o_means = take(sizeof(double) * (size_t)vk::logsum_scratch(D, S));
    const size_t o_delta = take(sizeof(double) * vk::kMaxS * kDim);
    const size_t o_dfix = take(sizeof(uint32_t) * vk::kMaxS * kDim);
    const size_t o_fbc = take(sizeof(int));
    const size_t fb_cap = mixed ? (size_t)D * groups + (size_t)vk::genz_items_slack(vk::device_sm_count(device)) : 1;
    const size_t o_fbi = take(sizeof(int2) * fb_cap);
    // parameter block, uploaded in one copy
    struct Params {
        ProbDev prob;
        ProbResult result;
        uint64_t seed;
        int32_t S;
        int32_t pad;
        int64_t off;
        int64_t means_off;
        int seg_prefix[2];
        int2 seg_base[1];
        uint32_t lattice[2 * kDim];
    };
    const size_t o_par = take(sizeof(Params));
    if (off > (size_t)VECCHIA_NOALLOC_SCRATCH_BYTES) return VECCHIA_ERR_UNSUPPORTED;

    unsigned char* base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc != VECCHIA_OK) return rc;

    Params h;
    std::memset(&h, 0, sizeof(h));
    rc = vecchia_lattice(N, kDim, h.lattice);
    if (rc != VECCHIA_OK) return rc;
    for (int j = 0; j < kDim; ++j)
        h.lattice[kDim + j] = (uint32_t)((((uint64_t)h.lattice[j] << 32) + (uint64_t)N / 2) / (uint64_t)N);
    Params* dpar = (Params*)(base + o_par);
    ProbDev& P = h.prob;
    P.sites = sites_ordered;
    P.nbr = nbr;
    P.u = u;
    P.num = (double*)(base + o_num);
    P.den = (double*)(base + o_den);
    P.g = dpar->lattice;
    P.gfix = dpar->lattice + kDim;
    P.delta = (const double*)(base + o_delta);
    P.dfix = (const uint32_t*)(base + o_dfix);
    P.D = D;
    P.n_terms = D;
    P.N = N;
    P.variance = cov.variance;
    P.range = cov.range;
    P.nu = cov.nu;
    P.nugget = cov.nugget;
    P.cov_kind = cov.kind;
    P.cos_a = (cov.kind == VECCHIA_COV_ANISO_EXP) ? std::cos(cov.angle) : 1.0;
    P.sin_a = (cov.kind == VECCHIA_COV_ANISO_EXP) ? std::sin(cov.angle) : 0.0;
    P.aspect = (cov.kind == VECCHIA_COV_ANISO_EXP) ? cov.aspect : 1.0;
    P.m = m;
    P.group = 0;
    P.S = S;
    P.dim = kDim;
    h.seed = seed;
    h.S = S;
    h.off = 0;
    h.means_off = 0;
    h.seg_prefix[0] = 0;
    h.seg_prefix[1] = (int)D;
    h.seg_base[0] = make_int2(0, 0);

    ProbResult res;
    int* fbc = (int*)(base + o_fbc);
    int2* fbi = (int2*)(base + o_fbi);
    cudaError_t e = cudaMemcpyAsync(dpar, &h, sizeof(Params), cudaMemcpyHostToDevice, st);
    // results and the flagged-site count start at zero on every call
    if (e == cudaSuccess) e = vk::launch_init_results(&dpar->result, 1, fbc, st);
    if (e == cudaSuccess)
        e = vk::launch_shifts(&dpar->seed, &dpar->S, &dpar->off, 1, kDim, (double*)(base + o_delta),
                              (uint32_t*)(base + o_dfix), st);
    if (e == cudaSuccess)
        e = vk::launch_genz(bucket, mixed, tile, &dpar->prob, dpar->seg_prefix, dpar->seg_base, 1, (int)D,
                            &dpar->result, fbc, fbi, S, (int)fb_cap, st);
    if (mixed && e == cudaSuccess)
        e = vk::launch_genz_fallback(bucket, &dpar->prob, fbc, fbi, (int)fb_cap, &dpar->result, S, st);
    if (e == cudaSuccess)
        e = vk::launch_logsum(&dpar->prob, 1, (int)vk::logsum_slices(D), &dpar->result, nullptr,
                              (double*)(base + o_means), &dpar->means_off, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&res, &dpar->result, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VECCHIA_ERR_CUDA;
    }
    if (res.status != VECCHIA_OK) return res.status;
    *log_p = res.log_p;
    *std_err = res.std_err;
    return VECCHIA_OK;
}
