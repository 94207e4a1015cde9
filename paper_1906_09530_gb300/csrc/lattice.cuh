// lattice.cuh -- D2Q9 velocity set (Sec. 2) and the BGK collision with
// exact-difference forcing (Eqs. 1, 2, 5), shared by the FP64 and FP32
// collide-stream kernels.
#pragma once

namespace cplbm {

// Velocity order of Sec. 2: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
// Called with compile-time i inside unrolled loops, so they fold to constants.
__host__ __device__ __forceinline__ constexpr int q_ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int q_ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

// Periodic index for v in [-1, n + 33), n >= 8 (tile halos): at most 5 steps.
__device__ __forceinline__ int wrap_near(int v, int n) {
    if (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// Explicitly rounded arithmetic.  With contraction left to the compiler, two
// inlined copies of the same formula in different contexts (the halo rows a
// collide-stream warp collides before its row loop, and the rows inside it) may
// be fused into multiply-adds differently and differ in the last bit, which
// would make results depend on the tile shape.  Every product, sum and fused
// multiply-add of the collision is therefore spelled out.
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }

// In-place BGK collision with exact-difference forcing:
//   f_i* = f_i - (f_i - f_i^eq(rho,u))/tau + [f_i^eq(rho,u+F/rho) - f_i^eq(rho,u)]
// With f_i^eq = w_i rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u) (c_s^2 = 1/3) and
// keep = 1 - 1/tau this is
//   f_i* = keep f_i + w_i rho [ (1-keep) - 3/2 (v.v - keep u.u)
//                               + 3 (e.v - keep e.u) + 9/2 ((e.v)^2 - keep (e.u)^2) ],
// v = u + F/rho.  Opposite directions share the even terms and flip the odd
// one, so each of the four pairs is evaluated once.  Returns false when rho is
// not a finite positive number.
template <typename T>
__device__ __forceinline__ bool collide_pairs(T f[9], T Fx, T Fy, T omega, T big) {
    const T rho = rn_add(rn_add(rn_add(rn_add(f[0], f[1]), rn_add(f[2], f[3])),
                                rn_add(rn_add(f[4], f[5]), rn_add(f[6], f[7]))),
                         f[8]);
    const T d57 = rn_sub(f[5], f[7]);
    const T jx = rn_add(rn_sub(f[1], f[3]), rn_add(d57, rn_sub(f[8], f[6])));
    const T jy = rn_add(rn_sub(f[2], f[4]), rn_add(d57, rn_sub(f[6], f[8])));
    const T inv = rn_div(T(1), rho);
    const T ux = rn_mul(jx, inv), uy = rn_mul(jy, inv);
    const T vx = rn_fma(Fx, inv, ux), vy = rn_fma(Fy, inv, uy);
    const T keep = rn_sub(T(1), omega);
    const T uu = rn_fma(ux, ux, rn_mul(uy, uy));
    const T vv = rn_fma(vx, vx, rn_mul(vy, vy));
    const T base = rn_fma(T(-1.5), rn_fma(-keep, uu, vv), omega);
    const T r0 = rn_mul(rho, T(4.0 / 9.0)), r1 = rn_mul(rho, T(1.0 / 9.0)),
            r2 = rn_mul(rho, T(1.0 / 36.0));
    f[0] = rn_fma(keep, f[0], rn_mul(r0, base));
    auto pair = [&](int i, int j, T w, T eu, T ev) {
        const T s = rn_fma(-keep, eu, ev);
        const T q = rn_fma(ev, ev, -rn_mul(keep, rn_mul(eu, eu)));
        const T A = rn_mul(w, rn_fma(T(4.5), q, base));
        const T B = rn_mul(w, rn_mul(T(3), s));
        f[i] = rn_fma(keep, f[i], rn_add(A, B));
        f[j] = rn_fma(keep, f[j], rn_sub(A, B));
    };
    pair(1, 3, r1, ux, vx);
    pair(2, 4, r1, uy, vy);
    pair(5, 7, r2, rn_add(ux, uy), rn_add(vx, vy));
    pair(6, 8, r2, rn_sub(uy, ux), rn_sub(vy, vx));
    return rho > T(0) && rho < big;
}

}  // namespace cplbm
