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

// ---- double-word numbers: an unevaluated sum h + l of two floats ----
// Built from the error-free transformations of Knuth (TwoSum) and Dekker (Fast2Sum, the
// exact product by FMA) and the double-word algorithms analysed by Joldes, Muller and
// Popescu (ACM TOMS 44, 2017): each operation below is exact to a few units of 2^-48
// relative, on the float32 pipe.
struct dw {
    float h, l;
};

// a + b = s + e exactly (any magnitudes)
__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// a + b = s + e exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a b = p + e exactly
__device__ __forceinline__ dw two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dw dw_from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dw_to(dw x) { return (double)x.h + (double)x.l; }
// x + y, renormalised
__device__ __forceinline__ dw dw_add(dw x, dw y) {
    dw s = two_sum(x.h, y.h);
    s.l = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
    return fast_two_sum(s.h, s.l);
}
// x - y (not renormalised: |l| stays within a few ulp of h)
__device__ __forceinline__ dw dw_sub(dw x, dw y) {
    dw s = two_sum(x.h, -y.h);
    s.l = __fadd_rn(s.l, __fsub_rn(x.l, y.l));
    return s;
}
// x y and x^2 (the l x l term, below 2^-48 relative, is dropped; not renormalised)
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    dw p = two_prod(x.h, y.h);
    p.l = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, p.l));
    return p;
}
__device__ __forceinline__ dw dw_sqr(dw x) {
    dw p = two_prod(x.h, x.h);
    p.l = __fmaf_rn(x.h, x.l, __fmaf_rn(x.h, x.l, p.l));
    return p;
}
// s += c k for non-negative terms; the low part gathers the product and sum errors and is
// left unnormalised (callers renormalise after a bounded number of terms)
__device__ __forceinline__ void dw_mac(dw& s, dw c, dw k) {
    const float p = __fmul_rn(c.h, k.h);
    float e = __fmaf_rn(c.h, k.h, -p);
    e = __fmaf_rn(c.h, k.l, e);
    e = __fmaf_rn(c.l, k.h, e);
    const dw t = two_sum(s.h, p);
    s.h = t.h;
    s.l = __fadd_rn(s.l, __fadd_rn(t.l, e));
}
__device__ __forceinline__ dw dw_renorm(dw x) { return fast_two_sum(x.h, x.l); }

// s += c k for non-negative c k and s: as dw_mac, with the running sum by Fast2Sum on the
// ordered pair (max, min) of the two high parts
__device__ __forceinline__ void dw_mac_pos(dw& s, dw c, dw k) {
    const float p = __fmul_rn(c.h, k.h);
    float e = __fmaf_rn(c.h, k.h, -p);
    e = __fmaf_rn(c.h, k.l, e);
    e = __fmaf_rn(c.l, k.h, e);
    const dw t = fast_two_sum(fmaxf(s.h, p), fminf(s.h, p));
    s.h = t.h;
    s.l = __fadd_rn(s.l, __fadd_rn(t.l, e));
}

// r2^e, e = -PW/4, for PW in {5, 6, 7} (2D kernels |x-y|^{-2-2s} of order s = 1/4, 1/2, 3/4)
// and PW in {1, 2, 3} (|x-y|^{-2s}, the strong form's single-layer kernel).  From the
// float32 estimate y0 of r2^{-1/2} (PW 2, 6) or r2^{-1/4} (PW 1, 3, 5, 7), about 2^-21
// relative: k0 = y0^m in double-word terms (m = 1, 3, 5, 7; built from the exact square of
// y0), then rho = 1 - r2 y0^2 (or 1 - r2 y0^4) from the same products, and
// k = k0 (1 - rho)^{-m/2 or -m/4} by the expansion to second order in rho (third-order
// terms are below 2^-56).  The float32 correction term is rounded once: about 2^-42 relative
// in the worst case, typically well below.
template <int PW>
__device__ __forceinline__ dw dw_kpow(dw x) {
    static_assert(PW == 1 || PW == 2 || PW == 3 || PW == 5 || PW == 6 || PW == 7,
                  "double-word powers: PW 1, 2, 3, 5, 6, 7");
    if constexpr (PW == 2 || PW == 6) {
        const float t0 = rsqrt_approx(x.h);
        const dw t2 = two_prod(t0, t0);
        const dw g = dw_mul(x, t2);  // x t0^2 ~ 1
        const float rho = __fsub_rn(__fsub_rn(1.f, g.h), g.l);
        dw k;
        float c;
        if constexpr (PW == 2) {
            k = {t0, 0.f};
            c = __fmul_rn(rho, __fmaf_rn(0.375f, rho, 0.5f));  // (1-rho)^{-1/2} - 1
        } else {
            k = two_prod(t2.h, t0);  // t0^3
            k.l = __fmaf_rn(t2.l, t0, k.l);
            c = __fmul_rn(rho, __fmaf_rn(1.875f, rho, 1.5f));  // (1-rho)^{-3/2} - 1
        }
        k.l = __fmaf_rn(k.h, c, k.l);
        return k;
    } else {
        const float v0 = rsqrt_approx(sqrt_approx(x.h));
        const dw v2 = two_prod(v0, v0);
        const dw v4 = dw_sqr(v2);
        const dw g = dw_mul(x, v4);  // x v0^4 ~ 1
        const float rho = __fsub_rn(__fsub_rn(1.f, g.h), g.l);
        dw k;
        float c;
        if constexpr (PW == 1) {
            k = {v0, 0.f};
            c = __fmul_rn(rho, __fmaf_rn(0.15625f, rho, 0.25f));  // (1-rho)^{-1/4} - 1
        } else if constexpr (PW == 3) {
            k = two_prod(v2.h, v0);  // v0^3
            k.l = __fmaf_rn(v2.l, v0, k.l);
            c = __fmul_rn(rho, __fmaf_rn(0.65625f, rho, 0.75f));  // (1-rho)^{-3/4} - 1
        } else if constexpr (PW == 5) {
            k = two_prod(v4.h, v0);  // v0^5
            k.l = __fmaf_rn(v4.l, v0, k.l);
            c = __fmul_rn(rho, __fmaf_rn(1.40625f, rho, 1.25f));  // (1-rho)^{-5/4} - 1
        } else {
            const dw v6 = dw_mul(v4, v2);
            k = two_prod(v6.h, v0);  // v0^7
            k.l = __fmaf_rn(v6.l, v0, k.l);
            c = __fmul_rn(rho, __fmaf_rn(2.40625f, rho, 1.75f));  // (1-rho)^{-7/4} - 1
        }
        k.l = __fmaf_rn(k.h, c, k.l);
        return k;
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace fl
