// df.cuh -- "double-float" arithmetic: a value carried as the unevaluated sum
// hi + lo of two floats (about 44-48 significant bits), built from the
// error-free transformations two-sum (Knuth) and fused multiply-add products.
// Every float operation is written with the _rn intrinsics so that the compiler
// cannot contract or reorder it (the error terms depend on exact rounding).
#pragma once

namespace cplbm {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df{-y.hi, -y.lo}); }
__device__ __forceinline__ df df_add_f(df x, float y) {
    const df s = two_sum(x.hi, y);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
// x * c for DF x and DF c (products by fmaf are exact error terms)
__device__ __forceinline__ df df_mul(df x, float ch, float cl) {
    const float p = __fmul_rn(x.hi, ch);
    float e = fmaf(x.hi, ch, -p);
    e = fmaf(x.hi, cl, e);
    e = fmaf(x.lo, ch, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ float df_round(df x) { return __fadd_rn(x.hi, x.lo); }

// x * c + y with the product left unnormalised before the sum (one
// renormalisation instead of two; same error bound to within a unit).
__device__ __forceinline__ df df_fma(df x, float ch, float cl, df y) {
    const float p = __fmul_rn(x.hi, ch);
    float e = fmaf(x.hi, ch, -p);
    e = fmaf(x.hi, cl, e);
    e = fmaf(x.lo, ch, e);
    const df s = two_sum(p, y.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, y.lo)));
}

// Exact sum of nine positive floats as a double-float, for populations whose
// largest member is normally f[0]: accumulating from f[0] with the exact
// a + b = s + e split (valid when |running sum| >= |addend|, so exact here
// whenever f[0] is the largest; otherwise an error of at most one unit of the
// low part).
__device__ __forceinline__ df sum9_exact(const float g[9]) {
    float s = g[0], e = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const float t = __fadd_rn(s, g[i]);
        e = __fadd_rn(e, __fsub_rn(g[i], __fsub_rn(t, s)));
        s = t;
    }
    return quick_two_sum(s, e);
}


}  // namespace cplbm
