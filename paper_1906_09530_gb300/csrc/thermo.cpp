// thermo.cpp -- host thermodynamics of the equations of state of Sec. 3.2
// needed to set up a run: the critical point (T_r = T/T_c) and the Maxwell
// coexistence densities (Sec. 5.1).
//
// Every EOS here has the form p0 = T A(rho) - alpha B(rho) (repulsion A,
// attraction B; alpha = 1 for CS and VDW, 1/sqrt(T) for RK, and the Soave or
// Peng-Robinson alpha(T_r), which is 1 at T_c, for RKS and PR):
//   CS   A = R rho Z(eta), eta = b rho/4          B = a rho^2              Eq. 20
//   VDW  A = R rho/(1 - b rho)                    B = a rho^2              Eq. 14
//   RK   A = R rho/(1 - b rho)                    B = a rho^2/(1 + b rho)  Eq. 16
//   PR   A = R rho/(1 - b rho)                    B = a rho^2/(1 + 2 b rho - b^2 rho^2)  Eq. 18
// On the spinodal dp0/drho = 0, so T A' = alpha B': T_sp(rho) = B'/A' (alpha = 1
// at criticality) or (B'/A')^(2/3) for RK.  The critical point is the maximum
// of T_sp over rho; there d2p0/drho2 = 0 as well, so B' A'' = B'' A' (for every
// kind), which fixes rho_c to rounding once the maximum is bracketed.
#include <cmath>

#include "cplbm_internal.cuh"

namespace cplbm {
namespace {

struct Eos {
    int kind;
    double a, b, R;
    bool cubic() const { return kind != LBM_EOS_CS; }
    double rho_max() const { return cubic() ? 1.0 / b : 4.0 / b; }
    // CS compressibility pieces (Eq. 20): d(rho Z)/d rho = H(eta)
    static double H(double e) {
        return (1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / std::pow(1 - e, 4);
    }
    double A(double r) const {
        if (!cubic()) {
            const double e = 0.25 * b * r;
            return R * r * (1 + e + e * e - e * e * e) / ((1 - e) * (1 - e) * (1 - e));
        }
        return R * r / (1 - b * r);
    }
    double dA(double r) const {
        if (!cubic()) return R * H(0.25 * b * r);
        return R / ((1 - b * r) * (1 - b * r));
    }
    static double dH(double e) {  // d H / d eta
        const double N = 1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e;
        const double dN = 4 + 8 * e - 12 * e * e + 4 * e * e * e;
        return (dN * (1 - e) + 4 * N) / std::pow(1 - e, 5);
    }
    double d2A(double r) const {
        if (!cubic()) return R * 0.25 * b * dH(0.25 * b * r);
        const double o = 1 - b * r;
        return 2 * R * b / (o * o * o);
    }
    double B(double r) const {
        switch (kind) {
            case LBM_EOS_RK:
            case LBM_EOS_RKS: return a * r * r / (1 + b * r);
            case LBM_EOS_PR: return a * r * r / (1 + 2 * b * r - b * b * r * r);
            default: return a * r * r;
        }
    }
    double dB(double r) const {
        switch (kind) {
            case LBM_EOS_RK:
            case LBM_EOS_RKS: return a * r * (2 + b * r) / ((1 + b * r) * (1 + b * r));
            case LBM_EOS_PR: {
                const double D = 1 + 2 * b * r - b * b * r * r;
                return a * (2 * r + 2 * b * r * r) / (D * D);
            }
            default: return 2 * a * r;
        }
    }
    double d2B(double r) const {
        switch (kind) {
            case LBM_EOS_RK:
            case LBM_EOS_RKS: {
                const double o = 1 + b * r;
                return 2 * a / (o * o * o);
            }
            case LBM_EOS_PR: {
                const double D = 1 + 2 * b * r - b * b * r * r;
                const double dD = 2 * b - 2 * b * b * r;
                return a * ((2 + 4 * b * r) * D - 2 * (2 * r + 2 * b * r * r) * dD) / (D * D * D);
            }
            default: return 2 * a;
        }
    }
    double t_spinodal(double r) const {
        const double q = dB(r) / dA(r);
        return kind == LBM_EOS_RK ? std::pow(q, 2.0 / 3.0) : q;
    }
};

// Temperature function alpha at T (RKS and PR need T_c; 1 at T = T_c).
double alpha_of(const Eos& e, double omega, double T, double Tc) {
    if (e.kind == LBM_EOS_RK) return 1.0 / std::sqrt(T);
    if (e.kind == LBM_EOS_RKS || e.kind == LBM_EOS_PR) {
        const double m = e.kind == LBM_EOS_RKS ? 0.480 + 1.574 * omega - 0.176 * omega * omega
                                               : 0.37464 + 1.54226 * omega -
                                                     0.26992 * omega * omega;
        const double s = 1 + m * (1 - std::sqrt(T / Tc));
        return s * s;
    }
    return 1.0;
}

struct State {
    Eos e;
    double T, al;
    double p0(double r) const { return T * e.A(r) - al * e.B(r); }
    double dp0(double r) const { return T * e.dA(r) - al * e.dB(r); }
    double mu0(double r) const {  // Eqs. 15, 17, 19, 21 without the gradient term
        const double a = e.a, b = e.b, R = e.R;
        switch (e.kind) {
            case LBM_EOS_CS: {
                const double x = 0.25 * b * r;
                return R * T * ((3 - x) / ((1 - x) * (1 - x) * (1 - x)) + std::log(r) + 1) -
                       2 * a * r;
            }
            case LBM_EOS_VDW:
                return R * T * (std::log(r / (1 - b * r)) + 1 / (1 - b * r)) - 2 * a * r;
            case LBM_EOS_RK:
            case LBM_EOS_RKS:
                return R * T * std::log(r / (1 - b * r)) + R * T / (1 - b * r) -
                       a * al / b * std::log(1 + b * r) - a * al * r / (1 + b * r);
            default: {
                const double s2 = std::sqrt(2.0);
                return R * T * std::log(r / (1 - b * r)) -
                       a * al / (2 * s2 * b) * std::log((s2 - 1 + b * r) / (s2 + 1 - b * r)) +
                       R * T / (1 - b * r) - a * al * r / (1 + 2 * b * r - b * b * r * r);
            }
        }
    }
};

// Bisection for a sign change of f on [lo, hi]; returns the midpoint of the
// final bracket.  f(lo) and f(hi) must differ in sign.
template <class F>
double bisect(F f, double lo, double hi, int iters = 200) {
    double flo = f(lo);
    for (int i = 0; i < iters; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = f(mid);
        if ((fm < 0) == (flo < 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

bool eos_ok(int kind, double a, double b, double R) {
    return kind >= LBM_EOS_CS && kind <= LBM_EOS_PR && a > 0 && b > 0 && R > 0;
}

}  // namespace

int eos_critical(int kind, double a, double b, double R, double* Tc, double* rhoc) {
    if (!eos_ok(kind, a, b, R)) return -1;
    const Eos e{kind, a, b, R};
    // golden-section search for the maximum of T_sp on (0, rho_max)
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double lo = 1e-6 * e.rho_max(), hi = 0.95 * e.rho_max();
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    double f1 = e.t_spinodal(x1), f2 = e.t_spinodal(x2);
    for (int i = 0; i < 200 && hi - lo > 1e-15 * e.rho_max(); ++i) {
        if (f1 < f2) {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + g * (hi - lo);
            f2 = e.t_spinodal(x2);
        } else {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - g * (hi - lo);
            f1 = e.t_spinodal(x1);
        }
    }
    // refine: B' A'' - B'' A' changes sign at rho_c
    const double r0 = 0.5 * (lo + hi);
    auto crit = [&](double r) { return e.dB(r) * e.d2A(r) - e.d2B(r) * e.dA(r); };
    double rc = r0;
    const double l2 = 0.9 * r0, h2 = std::fmin(1.1 * r0, 0.99 * e.rho_max());
    if ((crit(l2) < 0) != (crit(h2) < 0)) rc = bisect(crit, l2, h2);
    *rhoc = rc;
    *Tc = e.t_spinodal(rc);
    return 0;
}

double eos_alpha(int kind, double a, double b, double R, double omega, double T) {
    double Tc, rc;
    if (eos_critical(kind, a, b, R, &Tc, &rc)) return NAN;
    return alpha_of(Eos{kind, a, b, R}, omega, T, Tc);
}

// Maxwell construction: equal chemical potential and equal pressure on the gas
// and liquid branches.  Parametrised by the liquid density: for each rho_l the
// gas density with the same mu0 is found on the gas branch (bisection in
// log rho), and rho_l is bisected until the two pressures agree.
int eos_maxwell(int kind, double a, double b, double R, double omega, double T,
                double* rho_g, double* rho_l) {
    double Tc, rc;
    if (eos_critical(kind, a, b, R, &Tc, &rc)) return -1;
    if (!(T > 0 && T < Tc)) return -1;
    const Eos eo{kind, a, b, R};
    const State s{eo, T, alpha_of(eo, omega, T, Tc)};
    const double rmax = eo.rho_max();
    // spinodals: dp0/drho < 0 between them, > 0 outside
    const double sg = bisect([&](double r) { return s.dp0(r); }, 1e-300, rc);
    const double sl = bisect([&](double r) { return s.dp0(r); }, rc, rmax * (1 - 1e-15));
    const double mu_top = s.mu0(sg);  // highest mu on the gas branch
    // gas density with mu0 = m (mu0 rises monotonically on (0, sg))
    auto gas_for_mu = [&](double m) {
        const double x = bisect([&](double ls) { return s.mu0(std::exp(ls)) - m; },
                                std::log(1e-300), std::log(sg));
        return std::exp(x);
    };
    // liquid density whose mu0 equals the gas-spinodal mu (upper end of the bracket)
    const double ltop = bisect([&](double r) { return s.mu0(r) - mu_top; }, sl,
                               rmax * (1 - 1e-15));
    auto dp = [&](double rl) { return s.p0(rl) - s.p0(gas_for_mu(s.mu0(rl))); };
    const double rl = bisect(dp, sl, ltop);
    *rho_l = rl;
    *rho_g = gas_for_mu(s.mu0(rl));
    return 0;
}

}  // namespace cplbm
