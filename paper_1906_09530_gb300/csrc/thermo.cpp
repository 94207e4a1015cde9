// thermo.cpp -- host thermodynamics of the Carnahan-Starling EOS (Eqs. 20-21)
// needed to set up a run: the critical point (T_r = T/T_c, Sec. 3.2) and the
// Maxwell coexistence densities (Sec. 5.1).
#include <cmath>

#include "cplbm_internal.cuh"

namespace cplbm {
namespace {

struct Cs {
    double a, b, R, T;
    double p0(double rho) const {  // Eq. 20
        const double e = 0.25 * b * rho;
        return rho * R * T * (1 + e + e * e - e * e * e) / ((1 - e) * (1 - e) * (1 - e)) -
               a * rho * rho;
    }
    double mu0(double rho) const {  // Eq. 21 without the gradient term
        const double e = 0.25 * b * rho;
        return R * T * ((3 - e) / ((1 - e) * (1 - e) * (1 - e)) + std::log(rho) + 1) -
               2 * a * rho;
    }
    // d p0 / d rho = R T H(eta) - 2 a rho, H = d(rho Z)/d rho
    double dp0(double rho) const { return R * T * H(0.25 * b * rho) - 2 * a * rho; }
    static double H(double e) {
        return (1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / std::pow(1 - e, 4);
    }
    static double dH(double e) {  // d H / d eta
        const double N = 1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e;
        const double dN = 4 + 8 * e - 12 * e * e + 4 * e * e * e;
        return (dN * (1 - e) + 4 * N) / std::pow(1 - e, 5);
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

}  // namespace

// The critical point is where dp0/drho and d2p0/drho2 vanish together.  With
// eta = b rho/4 these read R T H(eta) = 8 a eta / b and R T H'(eta) = 8 a / b,
// so eta_c solves H(eta) = eta H'(eta) (independent of a, b, R), then
// T_c = 8 a / (b R H'(eta_c)) and rho_c = 4 eta_c / b.
int cs_critical(double a, double b, double R, double* Tc, double* rhoc) {
    if (!(a > 0 && b > 0 && R > 0)) return -1;
    auto g = [](double e) { return Cs::H(e) - e * Cs::dH(e); };
    const double ec = bisect(g, 0.01, 0.5);
    *Tc = 8 * a / (b * R * Cs::dH(ec));
    *rhoc = 4 * ec / b;
    return 0;
}

// Maxwell construction: equal chemical potential and equal pressure on the gas
// and liquid branches.  Parametrised by the liquid density: for each rho_l the
// gas density with the same mu0 is found on the gas branch (bisection in
// log rho), and rho_l is bisected until the two pressures agree.
int cs_maxwell(double a, double b, double R, double T, double* rho_g, double* rho_l) {
    double Tc, rc;
    if (cs_critical(a, b, R, &Tc, &rc)) return -1;
    if (!(T > 0 && T < Tc)) return -1;
    const Cs e{a, b, R, T};
    const double rmax = 4.0 / b;
    // spinodals: dp0/drho < 0 between them, > 0 outside
    const double sg = bisect([&](double r) { return e.dp0(r); }, 1e-300, rc);
    const double sl = bisect([&](double r) { return e.dp0(r); }, rc, rmax * (1 - 1e-15));
    const double mu_top = e.mu0(sg);  // highest mu on the gas branch
    // gas density with mu0 = m (mu0 rises monotonically on (0, sg))
    auto gas_for_mu = [&](double m) {
        const double s = bisect([&](double ls) { return e.mu0(std::exp(ls)) - m; },
                                std::log(1e-300), std::log(sg));
        return std::exp(s);
    };
    // liquid density whose mu0 equals the gas-spinodal mu (upper end of the bracket)
    const double ltop = bisect([&](double r) { return e.mu0(r) - mu_top; }, sl,
                               rmax * (1 - 1e-15));
    auto dp = [&](double rl) { return e.p0(rl) - e.p0(gas_for_mu(e.mu0(rl))); };
    const double rl = bisect(dp, sl, ltop);
    *rho_l = rl;
    *rho_g = gas_for_mu(e.mu0(rl));
    return 0;
}

}  // namespace cplbm
