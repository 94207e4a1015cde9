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
    const T rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const T jx = (f[1] - f[3]) + ((f[5] - f[7]) + (f[8] - f[6]));
    const T jy = (f[2] - f[4]) + ((f[5] - f[7]) + (f[6] - f[8]));
    const T inv = T(1) / rho;
    const T ux = jx * inv, uy = jy * inv;
    const T vx = ux + Fx * inv, vy = uy + Fy * inv;
    const T keep = T(1) - omega;
    const T base = omega - T(1.5) * ((vx * vx + vy * vy) - keep * (ux * ux + uy * uy));
    const T r0 = rho * T(4.0 / 9.0), r1 = rho * T(1.0 / 9.0), r2 = rho * T(1.0 / 36.0);
    f[0] = keep * f[0] + r0 * base;
    auto pair = [&](int i, int j, T w, T eu, T ev) {
        const T s = ev - keep * eu;
        const T q = ev * ev - keep * (eu * eu);
        const T A = w * (base + T(4.5) * q);
        const T B = w * (T(3) * s);
        f[i] = keep * f[i] + (A + B);
        f[j] = keep * f[j] + (A - B);
    };
    pair(1, 3, r1, ux, vx);
    pair(2, 4, r1, uy, vy);
    pair(5, 7, r2, ux + uy, vx + vy);
    pair(6, 8, r2, uy - ux, vy - vx);
    return rho > T(0) && rho < big;
}

}  // namespace cplbm
