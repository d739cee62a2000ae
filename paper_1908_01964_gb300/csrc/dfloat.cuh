// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi) / 2), about 48 significand bits, on the FP32 pipe.
// Used where a per-row quantity must be accurate beyond FP32 and FP64 would sit
// on a row's critical path (on sm_103a an FP64 warp instruction occupies its
// sub-partition's FP64 pipe for tens of cycles).  Error-free transformations:
//   two_sum       Knuth (The Art of Computer Programming, vol. 2, 4.2.2):
//                 s = fl(a + b) and the exact rounding error, for any a, b;
//   fast_two_sum  Dekker (1971), the same when |a| >= |b|;
//   two_prod      the exact error of fl(a * b) is fma(a, b, -fl(a * b)).
// Sums and products of double-floats follow Dekker's construction (1971): the
// leading terms exactly, the trailing terms in FP32, then renormalisation.
// Division and square root take an FP32 first approximation (IEEE division,
// sqrtf) and one Newton correction computed with the exact residual.
#pragma once

#include <cuda_runtime.h>

namespace rcscm {

struct df {
    float hi, lo;
};
struct dfc {   // complex double-float
    df re, im;
};

__device__ __forceinline__ df df_make(float v) { return df{v, 0.f}; }
__device__ __forceinline__ df df_from_double(double v) {
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
}
__device__ __forceinline__ float df_to_float(df x) { return x.hi + x.lo; }

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = a + b;
    return df{s, b - (s - a)};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = a * b;
    return df{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ df df_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}
// x / y: q = hi / hi, then q + (x - q y) / y with the residual formed exactly.
__device__ __forceinline__ df df_div(df x, df y) {
    const float q1 = x.hi / y.hi;
    const df r = df_sub(x, df_mul(df_make(q1), y));
    const float q2 = r.hi / y.hi;
    return fast_two_sum(q1, q2);
}
// sqrt(x), x >= 0: s = sqrtf(hi), then s + (x - s^2) / (2 s).
__device__ __forceinline__ df df_sqrt(df x) {
    if (!(x.hi > 0.f)) return df{0.f, 0.f};
    const float s = sqrtf(x.hi);
    const df r = df_sub(x, two_prod(s, s));
    return fast_two_sum(s, r.hi / (2.f * s));
}

__device__ __forceinline__ dfc dfc_make(df re, df im) { return dfc{re, im}; }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return dfc{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return dfc{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
    return dfc{df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// conj(a) * b
__device__ __forceinline__ dfc dfc_mulc(dfc a, dfc b) {
    return dfc{df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_sub(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dfc dfc_scale(dfc a, df s) { return dfc{df_mul(a.re, s), df_mul(a.im, s)}; }
__device__ __forceinline__ df dfc_abs2(dfc a) { return df_add(df_mul(a.re, a.re), df_mul(a.im, a.im)); }
__device__ __forceinline__ float2 dfc_to_float2(dfc a) { return make_float2(df_to_float(a.re), df_to_float(a.im)); }

}  // namespace rcscm
