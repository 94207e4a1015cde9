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


}  // namespace cplbm
