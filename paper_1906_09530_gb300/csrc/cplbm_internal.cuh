// cplbm_internal.cuh -- shared declarations of the CUDA library (device
// kernels, launchers and the context).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/cplbm.h"

namespace cplbm {

// Device-resident state block (one per context, inside the workspace).
struct DevState {
    int64_t t;              // time level of the populations in f[cur]
    unsigned int flag;      // error bits, see FLAG_*
    unsigned int pad0;
    unsigned long long failed_t;  // smallest flagged time level (ULLONG_MAX: none)
    double diag[4];         // mass, max|v|, rho_min, rho_max
};

enum : unsigned int {
    FLAG_RHO = 1u,   // collide-stream: rho <= 0 or not finite
    FLAG_EOS = 2u,   // EOS pass: b rho / 4 >= 1 (the CS pole) or mu not finite
};

// Compact-FD coefficients in the factorised form used by the line sweeps.
// The periodic system alpha d[i-1] + d[i] + alpha d[i+1] = (B u)[i] is split as
// A = (alpha/lam)(1 + lam S^-1)(1 + lam S), lam = (1 - sqrt(1 - 4 alpha^2))/(2 alpha),
// so d = (lam/alpha) (1 + lam S)^-1 (1 + lam S^-1)^-1 B u.  The factor lam/alpha
// is folded into the right-hand-side weights c1 = (lam/alpha) a/2 and
// c2 = (lam/alpha) b/4 (a, b from Eq. 38).  Each first-order recursion is cut
// after `warm` terms, where its weight has fallen below FP64 rounding.
struct CfdCoef {
    double c1, c2, lam;
    int warm;
    int sixth;  // 1 when b != 0 (the +-2 neighbours enter)
};

CfdCoef make_cfd_coef(int fd_order);

// Physical parameters the kernels need.
struct PhysParams {
    double T, a, b, R;   // EOS (Eq. 20), T absolute
    double k2;           // k^2 (Eq. 33)
    double kappa;        // kappa-hat (Eq. 33)
    double omega;        // 1 / tau (Eq. 1)
    double mu_cap;       // k^2 * mu_max (mesh-space limit, Sec. 5.6)
    int64_t cap_steps;   // limit active while t < cap_steps
};

// Launchers (all asynchronous on `s`).  Fields are FP64 [ny][nx]; populations
// are [9][plane] of TF with plane >= nx*ny.
template <typename TF>
cudaError_t launch_collide_stream(const TF* fin, TF* fout, const double* Fx, const double* Fy,
                                  double* rho_out, int nx, int ny, size_t plane, double omega,
                                  DevState* st, cudaStream_t s);

template <typename TF>
cudaError_t launch_init_feq(const double* rho, const double* ux, const double* uy, TF* f,
                            double* rho_out, int nx, int ny, size_t plane, cudaStream_t s);

template <typename TF>
cudaError_t launch_rho_from_f(const TF* f, double* rho, int nx, int ny, size_t plane,
                              cudaStream_t s);

template <typename TF>
cudaError_t launch_macro(const TF* f, const double* Fx, const double* Fy, double* vx,
                         double* vy, int nx, int ny, size_t plane, cudaStream_t s);

template <typename TF>
cudaError_t launch_diag(const TF* f, const double* rho, const double* Fx, const double* Fy,
                        int nx, int ny, size_t plane, double* partials, int nparts,
                        DevState* st, cudaStream_t s);

template <typename TF>
cudaError_t launch_f_to_double(const TF* f, double* out, size_t n, cudaStream_t s);
template <typename TF>
cudaError_t launch_f_from_double(const double* in, TF* f, size_t n, cudaStream_t s);

// Force stage (passes 2-5).
cudaError_t launch_cfd_x_rho(const double* rho, double* dxr, double* dxx, int nx, int ny,
                             int seg, const CfdCoef& c, DevState* st, int bump,
                             cudaStream_t s);
cudaError_t launch_cfd_y_rho_mu(const double* rho, const double* dxx, double* dyr, double* mu,
                                int nx, int ny, int seg, const CfdCoef& c,
                                const PhysParams& p, DevState* st, cudaStream_t s);
cudaError_t launch_cfd_x_force(const double* mu, const double* rho, const double* dxr,
                               double* Fx, int nx, int ny, int seg, const CfdCoef& c,
                               cudaStream_t s);
cudaError_t launch_cfd_y_force(const double* mu, const double* rho, const double* dyr,
                               double* Fy, int nx, int ny, int seg, const CfdCoef& c,
                               cudaStream_t s);
// Plain derivative(s) along an axis (stand-alone entry point).
cudaError_t launch_cfd_plain(const double* u, double* d1, double* d2, int nx, int ny, int axis,
                             int seg, const CfdCoef& c, cudaStream_t s);

int default_segment(int line_len, int n_lines);

// Host thermodynamics of the product library (independent of the oracle).
int cs_critical(double a, double b, double R, double* Tc, double* rhoc);
int cs_maxwell(double a, double b, double R, double T, double* rho_g, double* rho_l);

}  // namespace cplbm
