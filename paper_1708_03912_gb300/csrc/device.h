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

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace fl
