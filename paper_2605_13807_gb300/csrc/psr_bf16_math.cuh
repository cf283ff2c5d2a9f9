// FP32 arithmetic of the BF16 tensor-core paths' epilogues: gates, GELU and
// the two-way conditional, in forms built on the approximate special-function
// units.  Internal to libpsr.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace psr {
namespace bf16m {

// Approximate-unit forms used only by the BF16 paths (every value they
// produce is rounded to BF16 before the next MMA, except the last layer's
// output and the scan carry, where the errors below stay far under the BF16
// rounding of the operands):
//   sigmoid(x) = 1/2 + 1/2 tanh(x/2) with tanh.approx.f32 (rel. err ~2^-11)
//   erf(u) for GELU: Abramowitz & Stegun, Handbook of Mathematical Functions,
//   formula 7.1.28: erf(u) = 1 - (1 + a1 u + ... + a6 u^6)^-16, u >= 0,
//   |error| <= 3e-7, with one approximate reciprocal.
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// AS7.1.28 coefficients a1..a6
#define PSR_AS7128_A1 0.0705230784f
#define PSR_AS7128_A2 0.0422820123f
#define PSR_AS7128_A3 0.0092705272f
#define PSR_AS7128_A4 0.0001520143f
#define PSR_AS7128_A5 0.0002765672f
#define PSR_AS7128_A6 0.0000430638f

// log P(s | .) from the logit difference with the fast exponential and
// logarithm (absolute error ~1e-7, far below the BF16 path's tolerance).
__device__ __forceinline__ float site_logp_fast(float d, int s, int forced) {
    if (forced >= 0) return (s == forced) ? 0.0f : -INFINITY;
    const float x = s ? -d : d;  // log P = -softplus(x)
    return -(fmaxf(x, 0.0f) + __logf(1.0f + __expf(-fabsf(x))));
}

// Packed two-site forms (FP32x2: each lane is an IEEE FP32 operation, so the
// results equal the scalar ones; one instruction serves two sites).
__device__ __forceinline__ float2 gelu_fast2(float2 x) {
    const float2 k = make_float2(0.70710678118654752f, 0.70710678118654752f);
    const float2 u = __fmul2_rn(make_float2(fabsf(x.x), fabsf(x.y)), k);
    float2 p = __ffma2_rn(make_float2(PSR_AS7128_A6, PSR_AS7128_A6), u,
                          make_float2(PSR_AS7128_A5, PSR_AS7128_A5));
    p = __ffma2_rn(p, u, make_float2(PSR_AS7128_A4, PSR_AS7128_A4));
    p = __ffma2_rn(p, u, make_float2(PSR_AS7128_A3, PSR_AS7128_A3));
    p = __ffma2_rn(p, u, make_float2(PSR_AS7128_A2, PSR_AS7128_A2));
    p = __ffma2_rn(p, u, make_float2(PSR_AS7128_A1, PSR_AS7128_A1));
    p = __ffma2_rn(p, u, make_float2(1.0f, 1.0f));
    p = __fmul2_rn(p, p);
    p = __fmul2_rn(p, p);
    p = __fmul2_rn(p, p);
    p = __fmul2_rn(p, p);
    const float2 e = make_float2(copysignf(1.0f - rcp_approx(p.x), x.x),
                                 copysignf(1.0f - rcp_approx(p.y), x.y));
    const float2 hx = __fmul2_rn(make_float2(0.5f, 0.5f), x);
    return __ffma2_rn(hx, e, hx);
}

// GELU for outputs that are rounded to BF16 right away (layers 0 and 1):
// GELU(x) ~= x/2 (1 + tanh(x (g1 + g3 s + g5 s^2))), s = min(x^2, 36), with
// (g1, g3, g5) fitted here to minimise the maximum error against the exact erf
// GELU (2.6e-5 in FP32 arithmetic; tanh.approx adds at most ~2.5e-4 |x|,
// below the BF16 rounding step 2^-8 |x| of an activation of that size).
#define PSR_GELU_G1 7.975078843e-01f
#define PSR_GELU_G3 3.700564602e-02f
#define PSR_GELU_G5 -3.515167885e-04f

__device__ __forceinline__ float2 gelu_bf16out2(float2 x) {
    float2 sq = __fmul2_rn(x, x);
    sq = make_float2(fminf(sq.x, 36.0f), fminf(sq.y, 36.0f));
    float2 p = __ffma2_rn(make_float2(PSR_GELU_G5, PSR_GELU_G5), sq, make_float2(PSR_GELU_G3, PSR_GELU_G3));
    p = __ffma2_rn(p, sq, make_float2(PSR_GELU_G1, PSR_GELU_G1));
    const float2 arg = __fmul2_rn(p, x);
    const float2 t = make_float2(tanh_approx(arg.x), tanh_approx(arg.y));
    const float2 hx = __fmul2_rn(make_float2(0.5f, 0.5f), x);
    return __ffma2_rn(hx, t, hx);
}

// Gate a = sigmoid(z + b_z) = 1/2 + 1/2 tanh((z + b_z)/2) and the scan input
// b = (1 - a)(h~ + b_h) for two sites; hbz2 = (b_z/2, b_z/2).
__device__ __forceinline__ void gates2(float2 z, float2 c, float2 hbz2, float2 bh2, float2 &a,
                                       float2 &b) {
    const float2 zz = __ffma2_rn(make_float2(0.5f, 0.5f), z, hbz2);
    const float2 t = make_float2(tanh_approx(zz.x), tanh_approx(zz.y));
    a = __ffma2_rn(make_float2(0.5f, 0.5f), t, make_float2(0.5f, 0.5f));
    const float2 cv = __fadd2_rn(c, bh2);
    b = __ffma2_rn(make_float2(-a.x, -a.y), cv, cv);
}

}  // namespace bf16m
}  // namespace psr
