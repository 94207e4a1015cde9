// eos.cuh -- the chemical potential without its gradient term, mu0(rho), of the
// equations of state of Sec. 3.2, for the device: Carnahan-Starling (Eq. 21),
// van der Waals (Eq. 15), Redlich-Kwong and its Soave form (Eq. 17), and
// Peng-Robinson (Eq. 19), each as printed.  Written with explicitly rounded
// operations, so every inlined copy gives the same bits.  `bad` is set where
// rho is not positive or reaches the repulsive pole (b rho/4 >= 1 for CS,
// b rho >= 1 for the cubic EOSs).
#pragma once

#include "cplbm_internal.cuh"
#include "lattice.cuh"

namespace cplbm {

__device__ __forceinline__ float rn_log(float x) { return logf(x); }
__device__ __forceinline__ double rn_log(double x) { return log(x); }

template <class T>
__device__ __forceinline__ T eos_mu0(const EosC<T>& e, T r, bool& bad) {
    if (e.kind == LBM_EOS_CS) {
        const T eta = rn_mul(e.b, r);  // e.b holds b/4
        const T om = rn_sub(T(1), eta);
        const T z = rn_add(rn_add(rn_div(rn_sub(T(3), eta), rn_mul(rn_mul(om, om), om)),
                                  rn_log(r)),
                           T(1));
        bad |= !(r > T(0) && eta < T(1));
        return rn_fma(e.rt, z, -rn_mul(e.a2, r));
    }
    const T br = rn_mul(e.b, r);
    const T om = rn_sub(T(1), br);
    bad |= !(r > T(0) && om > T(0));
    const T lr = rn_log(rn_div(r, om));  // ln(rho / (1 - b rho))
    const T inv = rn_div(T(1), om);      // 1 / (1 - b rho)
    if (e.kind == LBM_EOS_VDW) return rn_fma(e.rt, rn_add(lr, inv), -rn_mul(e.a2, r));
    T m = rn_fma(e.rt, lr, rn_mul(e.rt, inv));
    if (e.kind == LBM_EOS_PR) {
        const T s2m = T(0.41421356237309515), s2p = T(2.414213562373095);
        const T lq = rn_log(rn_div(rn_add(s2m, br), rn_sub(s2p, br)));
        const T den = rn_sub(rn_fma(T(2), br, T(1)), rn_mul(br, br));  // 1 + 2 b rho - b^2 rho^2
        m = rn_sub(m, rn_mul(e.clog, lq));
        return rn_sub(m, rn_div(rn_mul(e.aal, r), den));
    }
    // RK and RKS
    m = rn_sub(m, rn_mul(e.clog, rn_log(rn_add(T(1), br))));
    return rn_sub(m, rn_div(rn_mul(e.aal, r), rn_add(T(1), br)));
}

// A positive density at or beyond the repulsive pole.  mu0 grows without bound
// as rho approaches the pole from below, so there it is +infinity: while the
// upper limit of Sec. 5.6 is active such a node takes the limit (the limit
// replaces the overflowing chemical potential); otherwise it is an error.
template <class T>
__device__ __forceinline__ bool eos_at_pole(const EosC<T>& e, T r) {
    return r > T(0) && rn_mul(e.b, r) >= T(1);  // e.b holds b/4 for CS
}

// mu-hat of the mixed path at one node: k^2 mu0(rho) - kappa (d_xx + d_yy) rho
// (Eq. 33 with the mu0 of Eqs. 15, 17, 19 or 21) in FP32, limited from above
// while the time level t < cap_steps (Sec. 5.6; `capped` comes from the time
// level read on the device, so that graph replays stay correct).  Shared by
// the lone and the batched pointwise kernels.
__device__ __forceinline__ float mu_node(float r, float xx, float yy, const MuConstF& p,
                                         bool capped, bool& bad) {
    bool b0 = false;
    const float mu0 = eos_mu0(p.e, r, b0);
    float m = rn_fma(p.k2, mu0, -rn_mul(p.kappa, rn_add(xx, yy)));
    if (capped) {
        if (eos_at_pole(p.e, r)) {  // mu0 = +infinity: the limit takes the node
            m = p.cap;
            b0 = false;
        } else {
            m = fminf(m, p.cap);
        }
    }
    bad |= b0 || !(fabsf(m) < 1e30f);
    return m;
}

}  // namespace cplbm
