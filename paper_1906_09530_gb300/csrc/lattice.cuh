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

// Opposite direction: e_opp(i) = -e_i.
__host__ __device__ __forceinline__ constexpr int q_opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
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
    T r0, r1, r2;
    if constexpr (sizeof(T) == 4) {
        // In FP32, 4/9, 1/9 and 1/36 share one mantissa and all round up by 7.5e-9.  Used as
        // constants, that bias adds mass every step and sets the populations' pressure apart
        // from the force's c_s^2 rho, which shifts the dilute gas at high density ratios.
        // Instead rho w_i = 16, 4, 1 x rho/36, with rho/36 = rho (hi + lo) rounded once.
        constexpr float hi = 1.0f / 36.0f;
        constexpr float lo = (float)(1.0 / 36.0 - (double)hi);
        r2 = rn_fma(rho, T(hi), rn_mul(rho, T(lo)));
        r1 = rn_mul(r2, T(4));
        r0 = rn_mul(r2, T(16));
    } else {
        r0 = rn_mul(rho, T(4.0 / 9.0));
        r1 = rn_mul(rho, T(1.0 / 9.0));
        r2 = rn_mul(rho, T(1.0 / 36.0));
    }
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

// MRT collision of Eq. 4 with exact-difference forcing (Eq. 5), in moment space:
//   m* = m - S (m - m^eq(u)) + [m^eq(u + F/rho) - m^eq(u)],   f* = M^-1 m*,
// on the standard D2Q9 basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy):
//   m^eq = (rho, rho(-2 + 3u.u), rho(1 - 3u.u), rho u_x, -rho u_x, rho u_y,
//           -rho u_y, rho(u_x^2 - u_y^2), rho u_x u_y),
// S = diag(0, s_e, s_eps, 0, s_q, 0, s_q, s_v, s_v), s_v = omega = 1/tau.  The
// forcing term, applied in velocity space as F_i = f^eq(v) - f^eq(u), is in
// moment space m^eq(v) - m^eq(u), because M is linear.  The rows of M are
// orthogonal, so M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
// Explicitly rounded, as collide_pairs.  Returns false when rho is not a finite
// positive number.
template <typename T>
__device__ __forceinline__ bool collide_mrt(T f[9], T Fx, T Fy, T omega, T big, T se, T seps,
                                            T sq) {
    const T s14 = rn_add(rn_add(f[1], f[2]), rn_add(f[3], f[4]));
    const T s58 = rn_add(rn_add(f[5], f[6]), rn_add(f[7], f[8]));
    const T rho = rn_add(rn_add(f[0], s14), s58);
    const T d57 = rn_sub(f[5], f[7]), d68 = rn_sub(f[6], f[8]);
    const T jx = rn_add(rn_sub(f[1], f[3]), rn_sub(d57, d68));
    const T jy = rn_add(rn_sub(f[2], f[4]), rn_add(d57, d68));
    const T inv = rn_div(T(1), rho);
    const T ux = rn_mul(jx, inv), uy = rn_mul(jy, inv);
    const T vx = rn_fma(Fx, inv, ux), vy = rn_fma(Fy, inv, uy);
    const T uu = rn_fma(ux, ux, rn_mul(uy, uy));
    const T vv = rn_fma(vx, vx, rn_mul(vy, vy));
    // moments of f
    const T e = rn_sub(rn_fma(T(2), s58, -s14), rn_mul(T(4), f[0]));
    const T eps = rn_add(rn_fma(T(-2), s14, s58), rn_mul(T(4), f[0]));
    const T qx = rn_add(rn_mul(T(2), rn_sub(f[3], f[1])), rn_sub(d57, d68));
    const T qy = rn_add(rn_mul(T(2), rn_sub(f[4], f[2])), rn_add(d57, d68));
    const T pxx = rn_sub(rn_add(f[1], f[3]), rn_add(f[2], f[4]));
    const T pxy = rn_sub(rn_add(f[5], f[7]), rn_add(f[6], f[8]));
    // relax toward m^eq(u), then add m^eq(v) - m^eq(u)
    const T dvu = rn_mul(T(3), rn_mul(rho, rn_sub(vv, uu)));
    const T e1 = rn_add(rn_fma(-se, rn_sub(e, rn_mul(rho, rn_fma(T(3), uu, T(-2)))), e), dvu);
    const T eps1 =
        rn_sub(rn_fma(-seps, rn_sub(eps, rn_mul(rho, rn_fma(T(-3), uu, T(1)))), eps), dvu);
    const T jx1 = rn_add(jx, rn_mul(rho, rn_sub(vx, ux)));
    const T jy1 = rn_add(jy, rn_mul(rho, rn_sub(vy, uy)));
    const T qx1 = rn_sub(rn_fma(-sq, rn_add(qx, jx), qx), rn_mul(rho, rn_sub(vx, ux)));
    const T qy1 = rn_sub(rn_fma(-sq, rn_add(qy, jy), qy), rn_mul(rho, rn_sub(vy, uy)));
    const T dxu = rn_fma(ux, ux, -rn_mul(uy, uy)), dxv = rn_fma(vx, vx, -rn_mul(vy, vy));
    const T pxx1 = rn_add(rn_fma(-omega, rn_sub(pxx, rn_mul(rho, dxu)), pxx),
                          rn_mul(rho, rn_sub(dxv, dxu)));
    const T xyu = rn_mul(ux, uy), xyv = rn_mul(vx, vy);
    const T pxy1 = rn_add(rn_fma(-omega, rn_sub(pxy, rn_mul(rho, xyu)), pxy),
                          rn_mul(rho, rn_sub(xyv, xyu)));
    // back to populations: f = M^T D^-1 m*
    const T a0 = rn_mul(rho, T(1.0 / 9.0)), a1 = rn_mul(e1, T(1.0 / 36.0)),
            a2 = rn_mul(eps1, T(1.0 / 36.0)), a3 = rn_mul(jx1, T(1.0 / 6.0)),
            a4 = rn_mul(qx1, T(1.0 / 12.0)), a5 = rn_mul(jy1, T(1.0 / 6.0)),
            a6 = rn_mul(qy1, T(1.0 / 12.0)), a7 = rn_mul(pxx1, T(0.25)),
            a8 = rn_mul(pxy1, T(0.25));
    const T c = rn_fma(T(-2), a2, rn_sub(a0, a1));          // a0 - a1 - 2 a2
    const T d = rn_add(rn_fma(T(2), a1, a0), a2);           // a0 + 2 a1 + a2
    const T x1 = rn_fma(T(-2), a4, a3), y1 = rn_fma(T(-2), a6, a5);
    const T x2 = rn_add(a3, a4), y2 = rn_add(a5, a6);
    f[0] = rn_fma(T(4), rn_sub(a2, a1), a0);
    f[1] = rn_add(rn_add(c, x1), a7);
    f[2] = rn_sub(rn_add(c, y1), a7);
    f[3] = rn_add(rn_sub(c, x1), a7);
    f[4] = rn_sub(rn_sub(c, y1), a7);
    f[5] = rn_add(rn_add(d, rn_add(x2, y2)), a8);
    f[6] = rn_sub(rn_add(d, rn_sub(y2, x2)), a8);
    f[7] = rn_add(rn_sub(d, rn_add(x2, y2)), a8);
    f[8] = rn_sub(rn_add(d, rn_sub(x2, y2)), a8);
    return rho > T(0) && rho < big;
}

}  // namespace cplbm
