// cov.cuh -- covariance functions of the spatial process (device), shared by
// the Vecchia kernel and the full-dimensional Genz path.  P is any struct with
// the fields cov_kind, variance, range, nu, cos_a, sin_a, aspect.
#pragma once

#include <cmath>

#include "vecchia.h"

namespace vk {

// Distance between two sites: Euclidean, or the Mahalanobis distance of
// Sec. 4.1 for the anisotropic exponential (explicit roundings, no contraction).
template <class P>
__device__ __forceinline__ double site_dist(const P& p, double dx, double dy) {
    if (p.cov_kind == VECCHIA_COV_ANISO_EXP) {
        const double o1 = __dsub_rn(__dmul_rn(dx, p.cos_a), __dmul_rn(dy, p.sin_a));
        const double o2 = __dmul_rn(p.aspect, __dadd_rn(__dmul_rn(dx, p.sin_a), __dmul_rn(dy, p.cos_a)));
        return sqrt(__dadd_rn(__dmul_rn(o1, o1), __dmul_rn(o2, o2)));
    }
    return sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// Exponential (and anisotropic exponential), or Matern with nu in {0.5, 1.5, 2.5}
// (Rasmussen-Williams form) at distance h.
__device__ __forceinline__ double cov_fn(int kind, double var, double range, double nu, double h) {
    if (kind != VECCHIA_COV_MATERN || nu == 0.5) return var * exp(-h / range);
    if (nu == 1.5) {
        const double a = 1.7320508075688772935 * h / range;
        return var * (1.0 + a) * exp(-a);
    }
    const double a = 2.2360679774997896964 * h / range;
    return var * (1.0 + a + a * a / 3.0) * exp(-a);
}

// Covariance parameters as the kernels read them (rotation precomputed).
struct CovParams {
    int cov_kind;
    double variance, range, nu, nugget, cos_a, sin_a, aspect;
};

inline CovParams cov_params(const vecchia_cov& c) {
    CovParams p;
    p.cov_kind = c.kind;
    p.variance = c.variance;
    p.range = c.range;
    p.nu = c.nu;
    p.nugget = c.nugget;
    p.cos_a = c.kind == VECCHIA_COV_ANISO_EXP ? std::cos(c.angle) : 1.0;
    p.sin_a = c.kind == VECCHIA_COV_ANISO_EXP ? std::sin(c.angle) : 0.0;
    p.aspect = c.kind == VECCHIA_COV_ANISO_EXP ? c.aspect : 1.0;
    return p;
}

}  // namespace vk
