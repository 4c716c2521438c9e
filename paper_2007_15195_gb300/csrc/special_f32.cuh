// special_f32.cuh -- generated by fit_special.py; do not edit by hand.
// Coefficients of the FP32 normal CDF / quantile pieces used by the mixed
// Genz kernel (forms and fitting method described in fit_special.py).
// Each piece: u = a*x + b maps its interval to [-1, 1]; value = sum_k c_k u^k.
#pragma once

namespace vk {
namespace special {

constexpr float kLog2e = 1.44269504088896341f;
constexpr float kKt = 3.535533906e-01f;  // t = 1 / (1 + z kKt)
constexpr float kZmax = 38.0f;

// PHI: log2 exponent; relative error of Phi; fit max error 7.38e-08, in float32 2.09e-07
constexpr float kPHIA = 2.148864586e+00f, kPHIB = -1.148864586e+00f;
constexpr int kPHIN = 10;
__device__ constexpr float kPHIC[10] = {-1.901662401e+00f, 9.110765296e-01f, 4.667263129e-02f, -5.721033787e-02f, -7.310898574e-03f, 9.311577214e-03f, 7.124167869e-04f, -1.848043810e-03f, 2.924683791e-06f, 2.557072991e-04f};

// INV1: f(w) = erfinv(y)/y on w in [0, 5]; fit max error 9.44e-08, in float32 2.02e-07
constexpr float kINV1A = 4.000000000e-01f, kINV1B = -1.000000000e+00f;
constexpr int kINV1N = 9;
__device__ constexpr float kINV1C[9] = {1.501409421e+00f, 6.166018141e-01f, -2.611067158e-02f, -1.958916803e-02f, 8.539142272e-03f, -4.294015403e-04f, -8.615332603e-04f, 2.098130980e-04f, 4.354054524e-05f};

// INV2: f(w) = erfinv(y)/y on s in [2.23607, 6]; fit max error 1.22e-07, in float32 2.37e-07
constexpr float kINV2A = 5.313592244e-01f, kINV2B = -2.188155346e+00f;
constexpr int kINV2N = 12;
__device__ constexpr float kINV2C[12] = {3.958954805e+00f, 1.900322869e+00f, 3.436654806e-03f, -4.783831998e-03f, 3.576914911e-03f, -2.687086927e-03f, 2.565709201e-04f, 3.193030862e-04f, 4.161732763e-03f, -4.454056890e-03f, -5.232413887e-04f, 1.333226713e-03f};

// INV3: f(w) = erfinv(y)/y on s in [6, 11.4018]; fit max error 7.02e-10, in float32 9.19e-08
constexpr float kINV3A = 3.702500904e-01f, kINV3B = -3.221500543e+00f;
constexpr int kINV3N = 9;
__device__ constexpr float kINV3C[9] = {8.583098189e+00f, 2.719722664e+00f, -3.118382403e-03f, 4.069332568e-04f, 2.902958468e-06f, -2.976520870e-05f, 1.599335430e-05f, -1.008701242e-05f, 4.181308814e-06f};

// INV4: f(w) = erfinv(y)/y on s in [11.4018, 26.4575]; fit max error 2.27e-10, in float32 1.62e-07
constexpr float kINV4A = 1.328395346e-01f, kINV4B = -2.514603728e+00f;
constexpr int kINV4N = 9;
__device__ constexpr float kINV4C[9] = {1.885506909e+01f, 7.547064667e+00f, -5.555254820e-03f, 1.660467877e-03f, -4.962391277e-04f, 1.464643870e-04f, -4.280124454e-05f, 9.922549798e-06f, -6.542327456e-07f};

}  // namespace special
}  // namespace vk
