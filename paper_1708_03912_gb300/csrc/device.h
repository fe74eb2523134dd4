// Device-side helpers shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fl {

// ---- fast float32 transcendental approximations (PTX approx instructions) ----
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// r2^e for the kernel |x-y|^{-d-2s} = (r2)^{e}, e = -(d+2s)/2.  PW selects an exact
// rewriting through square roots when 4e is an integer in -7..-3 (t = r2^{-1/2}):
//   PW=3: t^{3/2}   PW=4: t^2   PW=5: t^{5/2}   PW=6: t^3   PW=7: t^{7/2};
// PW=0 is the general power.
template <int PW>
__device__ __forceinline__ double kpow(double r2, double e) {
    if constexpr (PW == 0) {
        return pow(r2, e);
    } else {
        double t = rsqrt(r2);
        if constexpr (PW == 3) return t * sqrt(t);
        if constexpr (PW == 4) return t * t;
        if constexpr (PW == 5) return t * t * sqrt(t);
        if constexpr (PW == 6) return t * t * t;
        if constexpr (PW == 7) return t * t * t * sqrt(t);
    }
}
template <int PW>
__device__ __forceinline__ float kpow(float r2, float e) {
    if constexpr (PW == 0) {
        return ex2_approx(e * lg2_approx(r2));
    } else {
        float t = rsqrt_approx(r2);
        if constexpr (PW == 3) return t * sqrt_approx(t);
        if constexpr (PW == 4) return t * t;
        if constexpr (PW == 5) return t * t * sqrt_approx(t);
        if constexpr (PW == 6) return t * t * t;
        if constexpr (PW == 7) return t * t * t * sqrt_approx(t);
    }
}

// ---- double-float arithmetic on the float32 pipe (float64 is ~1/64 of its rate here) ----
// x = hi + lo + O(2^-47 |x|) with integer operations only (no float64 pipe): hi keeps
// the leading 24 significand bits (truncated), lo is the float32 value of the 29 bits
// dropped.  |x| < 2^-126 gives (0, 0); lo is dropped below 2^-74 |x|'s scale.
__device__ __forceinline__ void df_split(double x, float2& v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ff);
    if (e <= 1023 - 127) {
        v = make_float2(0.f, 0.f);
        return;
    }
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    if (e >= 1023 + 128) {  // beyond float32: an infinity that poisons the residual visibly
        v = make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
        return;
    }
    const unsigned long long m = u & ((1ull << 52) - 1);
    const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
    // dropped bits have weight 2^(e - 1023 - 52); as a float32 scale that needs e >= 949
    float lo = 0.f;
    if (e >= 1023 - 74) {
        const float scale = __uint_as_float((unsigned)(e - 1023 - 52 + 127) << 23);
        lo = __uint2float_rn((unsigned)(m & 0x1FFFFFFFu)) * scale;
        if (sign) lo = -lo;
    }
    v = make_float2(hi, lo);
}

// (sh, sl) += (ah + al)(uh + ul), dropping al ul
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float uh, float ul) {
    const float p = __fmul_rn(ah, uh);
    const float e = __fmaf_rn(ah, uh, -p);
    const float l = __fmaf_rn(ah, ul, __fmaf_rn(al, uh, e));
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, l));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace fl
