// f32x2.h -- packed pairs of FP32 values for the sm_100-family f32x2
// instructions (add/sub/mul/fma .f32x2, PTX ISA 8.6+).
//
// A pair is one 64-bit register holding two independent FP32 values (the two
// lattice points a lane evaluates).  One packed instruction does the work of
// two scalar ones with the same rounding (.rn, each element rounded as the
// scalar operation rounds it), so a packed evaluation is bit-identical to the
// scalar one while taking half the issue slots; the FMA pipe's throughput in
// lane operations is unchanged.
#pragma once

#include <stdint.h>

namespace vk {
namespace x2 {

typedef unsigned long long f2;

__device__ __forceinline__ f2 pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// The same value in both elements (an immediate when c is a constant).
__device__ __forceinline__ f2 splat(float c) {
    const unsigned long long b = __float_as_uint(c);
    return (b << 32) | b;
}
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Polynomial sum_k c_k u^k by Horner's rule on both elements (the scalar
// horner() of special_f32.h, element by element).
template <int N>
__device__ __forceinline__ f2 horner(const float (&c)[N], f2 u) {
    f2 acc = splat(c[N - 1]);
#pragma unroll
    for (int k = N - 2; k >= 0; --k) acc = fma(acc, u, splat(c[k]));
    return acc;
}

}  // namespace x2
}  // namespace vk
