// Double-float ("df") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits built from FP32 operations only.  Ray set-up
// (direction, entry point, per-brick sample ranges) runs in df so that FP32
// sample positions deep inside a large cube stay within ~1e-5 voxel of the
// exact ones without FP64, which is slow on this GPU.
//
// The error-free transformations are Knuth's TwoSum, Dekker's FastTwoSum and
// the FMA-based TwoProd; division and square root take one Newton correction.
// They rely on IEEE round-to-nearest FP32 without reassociation (no fast-math).
#pragma once
#include <cuda_runtime.h>

namespace vr {

struct df {
    float hi, lo;
};

__host__ __device__ inline df df_make(float hi, float lo = 0.0f) { return df{hi, lo}; }

// Split a host double into hi + lo.
__host__ inline df df_from_double(double x) {
    float hi = (float)x;
    float lo = (float)(x - (double)hi);
    return df{hi, lo};
}

__device__ __forceinline__ df df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    df t = df_two_sum(a.lo, b.lo);
    float e = __fadd_rn(s.lo, t.hi);
    s = df_fast_two_sum(s.hi, e);
    e = __fadd_rn(s.lo, t.lo);
    return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = df_two_sum(a.hi, b);
    float e = __fadd_rn(s.lo, a.lo);
    return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_fast_two_sum(p, e);
}

// a / b with two quotient corrections.
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_sub(a, df_mul_f(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_sub(r, df_mul_f(b, q2));
    float q3 = __fdiv_rn(r.hi, b.hi);
    df q = df_fast_two_sum(q1, q2);
    return df_add_f(q, q3);
}

__device__ __forceinline__ df df_sqrt(df a) {
    if (a.hi <= 0.0f) return df{0.0f, 0.0f};
    float s = __fsqrt_rn(a.hi);
    df r = df_sub(a, df_mul(df{s, 0.0f}, df{s, 0.0f}));
    float e = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
    return df_fast_two_sum(s, e);
}

__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_gt(df a, df b) { return df_lt(b, a); }
__device__ __forceinline__ df df_max(df a, df b) { return df_lt(a, b) ? b : a; }
__device__ __forceinline__ df df_min(df a, df b) { return df_lt(a, b) ? a : b; }
__device__ __forceinline__ bool df_is_zero(df a) { return a.hi == 0.0f; }
__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }

// floor / ceil of hi + lo as a float (exact integers below 2^24).
__device__ __forceinline__ float df_floor(df a) {
    float f = floorf(a.hi);
    if (f == a.hi) return a.lo < 0.0f ? f - 1.0f : f;
    return f;
}

__device__ __forceinline__ float df_ceil(df a) {
    float c = ceilf(a.hi);
    if (c == a.hi) return a.lo > 0.0f ? c + 1.0f : c;
    return c;
}

}  // namespace vr
