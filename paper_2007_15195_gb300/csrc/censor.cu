// censor.cu -- the conditional law of censored sites given observed ones, for
// the censored likelihood G_I of Sec. 4 (Eq. model05): with L the Cholesky
// factor of Sigma_II (observed sites I),
//   V_a = L^-1 Sigma_{I a}  (each censored site a),   w = L^-1 x_I,
//   mean_a = Sigma_{a I} Sigma_II^-1 x_I = V_a . w,
//   (Sigma_{c|I})_{ab} = Sigma_ab - V_a . V_b,
// so the Vecchia terms of the censored sites need only V (the Genz kernel
// subtracts V_a . V_b from each block entry) and the thresholds x_c - mean.
#include "cov.cuh"
#include "vk_internal.h"

namespace vk {
namespace {

// Forward substitution per row, one thread each: rows a < nc solve
// L v = Sigma_{I a}, row nc solves L w = x_I; each entry takes its terms in
// ascending order with fma, then the pivot division.
__global__ void cond_solve_kernel(const double* __restrict__ L, int k, const double* __restrict__ sites_i,
                                  const double* __restrict__ x_i, const double* __restrict__ sites_c, int nc,
                                  CovParams cv, double* __restrict__ V) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a > nc) return;
    double* row = V + (int64_t)a * k;
    for (int t = 0; t < k; ++t) {
        double acc;
        if (a < nc) {
            const double h = site_dist(cv, __dsub_rn(sites_i[2 * t], sites_c[2 * a]),
                                       __dsub_rn(sites_i[2 * t + 1], sites_c[2 * a + 1]));
            acc = cov_fn(cv.cov_kind, cv.variance, cv.range, cv.nu, h);
        } else {
            acc = x_i[t];
        }
        for (int s = 0; s < t; ++s) acc = fma(-L[(int64_t)t * k + s], row[s], acc);
        row[t] = acc / L[(int64_t)t * k + t];
    }
}

__global__ void cond_mean_kernel(const double* __restrict__ V, int k, int nc, const double* __restrict__ x_c,
                                 double* __restrict__ u_out) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nc) return;
    const double* va = V + (int64_t)a * k;
    const double* w = V + (int64_t)nc * k;
    double mu = 0.0;
    for (int t = 0; t < k; ++t) mu = fma(va[t], w[t], mu);
    u_out[a] = x_c[a] - mu;
}

}  // namespace

cudaError_t launch_conditioning(const double* L, int k, const double* sites_i, const double* x_i,
                                const double* sites_c, const double* x_c, int64_t nc, const vecchia_cov& cov,
                                double* V, double* u_out, cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    cond_solve_kernel<<<(unsigned)((nc + 1 + 127) / 128), 128, 0, st>>>(L, k, sites_i, x_i, sites_c, (int)nc,
                                                                        cov_params(cov), V);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && nc > 0) {
        cond_mean_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(V, k, (int)nc, x_c, u_out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace vk
