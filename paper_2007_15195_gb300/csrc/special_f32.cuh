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

// INV1 from L = log2(r (1-r)): u = kINV1LA L + kINV1LB, valid for L > kINV1Lmin
constexpr float kINV1LA = -1.732867951e-01f, kINV1LB = -1.346573590e+00f, kINV1Lmin = -1.354156033e+01f;

// INV1S from L' = log2(256 r (1-r)), Horner in L' itself, valid for L' > kINV1SLmin
constexpr float kINV1SLmin = -6.0f;

// PHI: log2 exponent as a polynomial in t itself; relative error of Phi; fit max error 7.38e-08, in float32 2.16e-07
constexpr float kPHIA = 1.000000000e+00f, kPHIB = 0.000000000e+00f;
constexpr int kPHIN = 10;
__device__ constexpr float kPHIC[10] = {-2.825746561e+00f, 1.442697133e+00f, 5.398850582e-01f, 1.395404485e-01f, -2.716838926e-01f, 4.150338577e-01f, -1.662797825e+00f, 2.173985704e+00f, -1.200732298e+00f, 2.498184801e-01f};

// INV1: sqrt(2) erfinv(y)/y on w in [0, 8]; fit max error 8.68e-08, in float32 1.93e-07
constexpr float kINV1A = 2.500000000e-01f, kINV1B = -1.000000000e+00f;
constexpr int kINV1N = 11;
__device__ constexpr float kINV1C[11] = {2.628710547e+00f, 1.291766786e+00f, -1.633898537e-01f, -1.841084796e-02f, 4.300585238e-02f, -2.277074509e-02f, 2.914623517e-03f, 4.860883741e-03f, -3.243484563e-03f, -1.816164950e-04f, 5.808041748e-04f};

// INV1S: sqrt(2) erfinv(y)/y / 16 as a polynomial in L' = log2(256 r (1-r)), w in [0, 8.31777]; fit max error 1.30e-07, in float32 2.96e-07
constexpr float kINV1SA = 1.000000000e+00f, kINV1SB = 0.000000000e+00f;
constexpr int kINV1SN = 11;
__device__ constexpr float kINV1SC[11] = {1.674851056e-01f, -1.384895821e-02f, -3.100284359e-04f, 3.872862671e-06f, 2.174756666e-06f, 2.151596011e-07f, 6.789406408e-09f, -1.169283648e-09f, -1.575603574e-10f, 2.953243844e-13f, 7.592575372e-13f};

// INV2: sqrt(2) erfinv(y)/y on s in [2.82843, 6]; fit max error 4.91e-08, in float32 1.41e-07
constexpr float kINV2A = 6.306019375e-01f, kINV2B = -2.783611625e+00f;
constexpr int kINV2N = 10;
__device__ constexpr float kINV2C[10] = {6.021852018e+00f, 2.265439361e+00f, 1.569894155e-03f, -2.705211631e-03f, 1.596556497e-03f, -7.857980017e-04f, 8.824118087e-06f, 4.160093507e-05f, 4.780434979e-04f, -3.270530312e-04f};

// INV3: sqrt(2) erfinv(y)/y on s in [6, 11.4018]; fit max error 7.02e-10, in float32 1.29e-07
constexpr float kINV3A = 3.702500904e-01f, kINV3B = -3.221500543e+00f;
constexpr int kINV3N = 9;
__device__ constexpr float kINV3C[9] = {1.213833387e+01f, 3.846268677e+00f, -4.410058687e-03f, 5.754905307e-04f, 4.105403236e-06f, -4.209436183e-05f, 2.261801856e-05f, -1.426518977e-05f, 5.913263633e-06f};

// INV4: sqrt(2) erfinv(y)/y on s in [11.4018, 26.4575]; fit max error 2.27e-10, in float32 1.21e-07
constexpr float kINV4A = 1.328395346e-01f, kINV4B = -2.514603728e+00f;
constexpr int kINV4N = 9;
__device__ constexpr float kINV4C[9] = {2.666509443e+01f, 1.067316121e+01f, -7.856316709e-03f, 2.348256191e-03f, -7.017881046e-04f, 2.071319224e-04f, -6.053010051e-05f, 1.403260450e-05f, -9.252248218e-07f};

}  // namespace special
}  // namespace vk
