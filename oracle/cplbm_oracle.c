/*
 * cplbm_oracle.c -- plain FP64 CPU oracle of the chemical-potential multiphase
 * lattice Boltzmann method of Wen, Zhao, Qiu, Ye and Shan (arXiv:1906.09530).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or constant with the CUDA library: every formula below is written out
 * again from the paper.
 *
 * It is deliberately slow and literal: plain nested loops, one time step in the
 * order the method states, cyclic tridiagonal systems solved by the Thomas
 * algorithm extended to periodic lines with the Sherman-Morrison formula.
 * Compiled with -ffp-contract=off so that x86 and Arm hosts give the same bits.
 *
 * Notation (mesh space, Sec. 4.1): grid step 1, time step 1, lattice c_s^2 = 1/3.
 *   k      proportional coefficient of Eq. 25 (mesh_coeff)
 *   kappa  the mesh-space kappa-hat of Eq. 33
 *   T      absolute temperature (T = T_r * T_c, Sec. 3.2)
 *   a,b,R  EOS constants (Carnahan-Starling, Eq. 20: the paper uses a=1, b=4, R=1)
 *   eos    0 CS (Eqs. 20-21), 1 VDW (Eqs. 14-15), 2 RK, 3 RKS (Eqs. 16-17),
 *          4 PR (Eqs. 18-19); eos_alpha the temperature function alpha(T) of
 *          RK/RKS/PR at the run's T (1 for CS and VDW)
 *
 * Populations are stored structure-of-arrays, f[i][y][x], i = 0..8 in the
 * velocity order of Sec. 2.
 *
 * Periodic in x; in y periodic or between solid walls (Sec. 5.5): halfway
 * bounce-back, walls that may move along x (a moving reference frame), and the
 * density and mu-hat extended evenly about the walls for their y-derivatives.
 * The chemical-potential upper limit of Sec. 5.6 also takes the EOS pole.
 *
 * Threads: built with OpenMP, the loops over lines and over nodes are shared
 * among orc_set_threads(n) threads (1 unless set).  Every line and every node is
 * computed exactly as with one thread, so the results do not depend on n.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 velocity set and weights, Sec. 2 (after Eq. 2). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 with c = 1 */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6}; /* e_OPP[i] = -e_i */

typedef struct {
    int32_t nx, ny;
    double T, a, b, R;      /* EOS (Eq. 20/21) */
    double kappa, tau, k;   /* kappa-hat (Eq. 33), BGK tau (Eq. 1), k (Eq. 25) */
    double alpha;           /* compact-FD alpha of Eq. 37/38: 1/4 (4th) or 1/3 (6th) */
    double mu_max;          /* chemical-potential upper limit (Sec. 5.6), momentum units */
    int64_t mu_cap_steps;   /* the limit acts while the time level t < mu_cap_steps */
    int32_t eos;            /* EOS kind, see the header comment (0: CS) */
    double eos_alpha;       /* alpha(T) of Eqs. 16-19 */
    int32_t mrt;            /* 0: BGK collision (Eq. 1); 1: MRT collision (Eq. 4) */
    double s[9];            /* MRT relaxation rates, the diagonal of S in Eq. 4 */
    int32_t walls_y;        /* 1: solid walls below y = 0 and above y = ny - 1 (Sec. 5.5) */
    double wall_ux[2];      /* x-velocity of the bottom and the top wall (0: at rest) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Equation of state                                                         */
/* ------------------------------------------------------------------------ */

/* Carnahan-Starling pressure, Eq. 20. */
double orc_cs_p0(double rho, double T, double a, double b, double R)
{
    double eta = b * rho / 4.0;
    double num = 1.0 + eta + eta * eta - eta * eta * eta;
    double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
    return rho * R * T * num / den - a * rho * rho;
}

/* Carnahan-Starling chemical potential without the gradient term, Eq. 21
 * (the psi'(rho) of Eq. 33), taken exactly as printed. */
double orc_cs_mu0(double rho, double T, double a, double b, double R)
{
    double eta = b * rho / 4.0;
    double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
    return R * T * ((3.0 - eta) / den + log(rho) + 1.0) - 2.0 * a * rho;
}

/* Pressure of each EOS of Sec. 3.2 as printed: VDW Eq. 14, RK/RKS Eq. 16,
 * PR Eq. 18, CS Eq. 20.  al is alpha(T) (unused by VDW and CS). */
double orc_p0(int kind, double rho, double T, double a, double b, double R, double al)
{
    if (kind == 0)
        return orc_cs_p0(rho, T, a, b, R);
    double rep = rho * R * T / (1.0 - b * rho);
    if (kind == 1)
        return rep - a * rho * rho;
    if (kind == 2 || kind == 3)
        return rep - a * al * rho * rho / (1.0 + b * rho);
    return rep - a * al * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* Chemical potential without the gradient term of each EOS as printed:
 * VDW Eq. 15, RK/RKS Eq. 17, PR Eq. 19, CS Eq. 21. */
double orc_mu0(int kind, double rho, double T, double a, double b, double R, double al)
{
    if (kind == 0)
        return orc_cs_mu0(rho, T, a, b, R);
    double om = 1.0 - b * rho;
    if (kind == 1)
        return R * T * (log(rho / om) + 1.0 / om) - 2.0 * a * rho;
    if (kind == 2 || kind == 3)
        return R * T * log(rho / om) + R * T / om - a * al / b * log(1.0 + b * rho) -
               a * al * rho / (1.0 + b * rho);
    double s2 = sqrt(2.0);
    return R * T * log(rho / om) -
           a * al / (2.0 * s2 * b) * log((s2 - 1.0 + b * rho) / (s2 + 1.0 - b * rho)) +
           R * T / om - a * al * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* ------------------------------------------------------------------------ */
/* Compact finite differences on a periodic line, Eqs. 37-38                 */
/* ------------------------------------------------------------------------ */

/* Thomas algorithm for a tridiagonal system with sub-diagonal lo[i] (row i,
 * column i-1), diagonal di[i] and super-diagonal up[i] (row i, column i+1).
 * cw is caller scratch of n doubles.  x may alias nothing else. */
static void thomas(int n, const double *lo, const double *di, const double *up,
                   const double *r, double *x, double *cw)
{
    double m = di[0];
    cw[0] = up[0] / m;
    x[0] = r[0] / m;
    for (int i = 1; i < n; ++i) {
        m = di[i] - lo[i] * cw[i - 1];
        cw[i] = up[i] / m;
        x[i] = (r[i] - lo[i] * x[i - 1]) / m;
    }
    for (int i = n - 2; i >= 0; --i)
        x[i] = x[i] - cw[i] * x[i + 1];
}

/* First derivative of the periodic samples u[0..n-1] (read with stride `su`,
 * spacing h) by the compact scheme of Eq. 37 with a and b from Eq. 38:
 *   alpha*d[i-1] + d[i] + alpha*d[i+1]
 *       = a*(u[i+1]-u[i-1])/(2h) + b*(u[i+2]-u[i-2])/(4h),   indices mod n.
 * The cyclic tridiagonal system is solved by the Thomas algorithm (Sec. 4.3)
 * extended to the periodic corners by the Sherman-Morrison formula.
 * The result goes to d (stride `sd`).  n >= 3.  Returns 0 or -1 (n < 3, no memory). */
int orc_cfd_line(const double *u, ptrdiff_t su, double *d, ptrdiff_t sd, int n,
                 double alpha, double h)
{
    if (n < 3)
        return -1;
    double ca = 2.0 / 3.0 * (alpha + 2.0);   /* Eq. 38 */
    double cb = (4.0 * alpha - 1.0) / 3.0;   /* Eq. 38 */
    double *buf = (double *)malloc(sizeof(double) * 8 * (size_t)n);
    if (!buf)
        return -1;
    double *r = buf, *lo = buf + n, *di = buf + 2 * n, *up = buf + 3 * n;
    double *y = buf + 4 * n, *z = buf + 5 * n, *uu = buf + 6 * n, *cw = buf + 7 * n;

    for (int i = 0; i < n; ++i) {
        int ip1 = (i + 1) % n, im1 = (i - 1 + n) % n;
        int ip2 = (i + 2) % n, im2 = (i - 2 + 2 * n) % n;
        r[i] = ca * (u[ip1 * su] - u[im1 * su]) / (2.0 * h) +
               cb * (u[ip2 * su] - u[im2 * su]) / (4.0 * h);
    }
    /* A = T' + w v^T with the corner entries A[0][n-1] = A[n-1][0] = alpha moved
     * into the rank-one term: w = (gamma,0,...,0,alpha), v = (1,0,...,0,alpha/gamma). */
    double gamma = -1.0;
    for (int i = 0; i < n; ++i) {
        lo[i] = alpha;
        di[i] = 1.0;
        up[i] = alpha;
        uu[i] = 0.0;
    }
    di[0] = 1.0 - gamma;
    di[n - 1] = 1.0 - alpha * alpha / gamma;
    uu[0] = gamma;
    uu[n - 1] = alpha;
    thomas(n, lo, di, up, r, y, cw);
    thomas(n, lo, di, up, uu, z, cw);
    double vy = y[0] + alpha / gamma * y[n - 1];
    double vz = z[0] + alpha / gamma * z[n - 1];
    double fac = vy / (1.0 + vz);
    for (int i = 0; i < n; ++i)
        d[i * sd] = y[i] - fac * z[i];
    free(buf);
    return 0;
}

/* Threads for the loops below (OpenMP builds; ignored otherwise). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* d/dx of a [ny][nx] field: every x-line in turn. */
static int cfd_x(const orc_params *p, const double *u, double *d)
{
    int err = 0;
#pragma omp parallel for reduction(| : err) schedule(static)
    for (int y = 0; y < p->ny; ++y)
        err |= orc_cfd_line(u + (size_t)y * p->nx, 1, d + (size_t)y * p->nx, 1, p->nx,
                            p->alpha, 1.0) != 0;
    return err ? -1 : 0;
}

/* d/dy of a [ny][nx] field: every y-line in turn. */
/* y-lines.  With walls, every field is extended evenly about both walls
 * (ghost y = -1 - j equals y = j, ghost y = ny + j equals y = ny - 1 - j): the
 * first ghost takes the value of its fluid neighbour, the wall rule of Sec. 5.5,
 * and the extended line is periodic with period 2 ny, so the same periodic
 * compact scheme applies; the first ny results are the derivatives. */
static int cfd_y(const orc_params *p, const double *u, double *d)
{
    int ny = p->ny;
    int err = 0;
    if (!p->walls_y) {
#pragma omp parallel for reduction(| : err) schedule(static)
        for (int x = 0; x < p->nx; ++x)
            err |= orc_cfd_line(u + x, p->nx, d + x, p->nx, ny, p->alpha, 1.0) != 0;
        return err ? -1 : 0;
    }
#pragma omp parallel reduction(| : err)
    {
        double *line = (double *)malloc(sizeof(double) * 4 * ny);
        if (!line)
            err = 1;
        double *dl = line ? line + 2 * ny : NULL;
#pragma omp for schedule(static)
        for (int x = 0; x < p->nx; ++x) {
            if (!line)
                continue;
            for (int y = 0; y < ny; ++y) {
                line[y] = u[(size_t)y * p->nx + x];
                line[2 * ny - 1 - y] = u[(size_t)y * p->nx + x];
            }
            err |= orc_cfd_line(line, 1, dl, 1, 2 * ny, p->alpha, 1.0) != 0;
            for (int y = 0; y < ny; ++y)
                d[(size_t)y * p->nx + x] = dl[y];
        }
        free(line);
    }
    return err ? -1 : 0;
}

/* d2/dy2 of a [ny][nx] field, "applying CFM twice" (Sec. 4.3) along the
 * line the field is extended to.  Periodic: cfd_y twice.  With walls the
 * density is what is extended evenly; the scheme is applied twice over the
 * whole period 2 ny, so the intermediate first derivative keeps the odd
 * symmetry the derivative of an even line has (it is not extended again). */
static int cfd_yy(const orc_params *p, const double *u, double *d)
{
    int ny = p->ny;
    if (!p->walls_y) {
        double *tmp = (double *)malloc(sizeof(double) * (size_t)p->nx * ny);
        if (!tmp)
            return -1;
        int err = cfd_y(p, u, tmp) | cfd_y(p, tmp, d);
        free(tmp);
        return err ? -1 : 0;
    }
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        double *line = (double *)malloc(sizeof(double) * 6 * ny);
        if (!line)
            err = 1;
        double *dl = line ? line + 2 * ny : NULL, *ddl = line ? line + 4 * ny : NULL;
#pragma omp for schedule(static)
        for (int x = 0; x < p->nx; ++x) {
            if (!line)
                continue;
            for (int y = 0; y < ny; ++y) {
                line[y] = u[(size_t)y * p->nx + x];
                line[2 * ny - 1 - y] = u[(size_t)y * p->nx + x];
            }
            err |= orc_cfd_line(line, 1, dl, 1, 2 * ny, p->alpha, 1.0) != 0;
            err |= orc_cfd_line(dl, 1, ddl, 1, 2 * ny, p->alpha, 1.0) != 0;
            for (int y = 0; y < ny; ++y)
                d[(size_t)y * p->nx + x] = ddl[y];
        }
        free(line);
    }
    return err ? -1 : 0;
}

/* The compact derivative of a whole field along x (axis 0) or y (axis 1), or
 * the second derivative along y (axis 2) as the force stage takes it, with the
 * run's boundaries; exported for the tests.  Returns 0 or -1. */
int orc_cfd_field(const orc_params *p, int axis, const double *u, double *d)
{
    return axis == 0 ? cfd_x(p, u, d) : axis == 1 ? cfd_y(p, u, d) : cfd_yy(p, u, d);
}

/* ------------------------------------------------------------------------ */
/* Lattice Boltzmann pieces                                                  */
/* ------------------------------------------------------------------------ */

/* Second-order equilibrium, Eq. 2. */
static double feq(int i, double rho, double ux, double uy)
{
    double eu = EX[i] * ux + EY[i] * uy;
    double uu = ux * ux + uy * uy;
    return WQ[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Exact-difference forcing term, Eq. 5 with delta-t = 1:
 *   F_i = f_i^eq(rho, u + F/rho) - f_i^eq(rho, u). */
void orc_forcing_terms(double rho, double ux, double uy, double Fx, double Fy, double *Fi)
{
    double dux = Fx / rho, duy = Fy / rho;
    for (int i = 0; i < 9; ++i)
        Fi[i] = feq(i, rho, ux + dux, uy + duy) - feq(i, rho, ux, uy);
}

/* Equilibrium populations for given rho, u (the initial state of a run). */
void orc_feq_field(const orc_params *p, const double *rho, const double *ux,
                   const double *uy, double *f)
{
    size_t N = (size_t)p->nx * p->ny;
    for (int i = 0; i < 9; ++i)
        for (size_t n = 0; n < N; ++n)
            f[i * N + n] = feq(i, rho[n], ux ? ux[n] : 0.0, uy ? uy[n] : 0.0);
}

/* Density and velocity moments, Eq. 3. */
static void moments(const orc_params *p, const double *f, double *rho, double *ux,
                    double *uy)
{
    size_t N = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            r += f[i * N + n];
            jx += EX[i] * f[i * N + n];
            jy += EY[i] * f[i * N + n];
        }
        rho[n] = r;
        ux[n] = jx / r;
        uy[n] = jy / r;
    }
}

/* The force stage at time level t, from rho alone:
 *   d_x rho, d_y rho                      compact FD, Eq. 39 (or its alpha family)
 *   d_xx rho = D_x(D_x rho), likewise y   "applying CFM twice", Sec. 4.3
 *                                         (with walls: along the extended line)
 *   mu-hat = k^2 mu0(rho) - kappa (d_xx rho + d_yy rho)          Eq. 33
 *            (mu0 = +infinity at or beyond the repulsive pole)
 *   mu-hat <- min(mu-hat, k^2 mu_max) while t < mu_cap_steps    Sec. 5.6
 *   F = -rho grad(mu-hat) + c_s^2 grad(rho)                     Eq. 12
 * Any output pointer may be NULL except Fx, Fy.  Returns 0 or -1. */
int orc_force_stage(const orc_params *p, int64_t t, const double *rho, double *mu_out,
                    double *Fx, double *Fy)
{
    size_t N = (size_t)p->nx * p->ny;
    double *buf = (double *)malloc(sizeof(double) * 7 * N);
    if (!buf)
        return -1;
    double *dxr = buf, *dyr = buf + N, *dxxr = buf + 2 * N, *dyyr = buf + 3 * N;
    double *mu = buf + 4 * N, *dxmu = buf + 5 * N, *dymu = buf + 6 * N;
    int err = 0;
    err |= cfd_x(p, rho, dxr);
    err |= cfd_y(p, rho, dyr);
    err |= cfd_x(p, dxr, dxxr);
    err |= cfd_yy(p, rho, dyyr);
    double k2 = p->k * p->k;
    /* the repulsive pole: b rho / 4 = 1 (CS, Eq. 21) or b rho = 1 (Eqs. 15-19) */
    double bpole = p->eos == 0 ? p->b / 4.0 : p->b;
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        /* mu0 grows without bound as rho approaches the pole from below; at or
         * beyond it mu0 is taken as that limit, +infinity (where the printed
         * formula has no real value, or for CS turns negative).  With the upper
         * limit active this gives k^2 mu_max (Sec. 5.6: the limit replaces the
         * overflowing chemical potential); without it the run fails there. */
        double m0 = rho[n] > 0.0 && bpole * rho[n] >= 1.0
                        ? INFINITY
                        : orc_mu0(p->eos, rho[n], p->T, p->a, p->b, p->R, p->eos_alpha);
        double m = k2 * m0 - p->kappa * (dxxr[n] + dyyr[n]);
        if (t < p->mu_cap_steps && m > k2 * p->mu_max)
            m = k2 * p->mu_max;
        mu[n] = m;
    }
    err |= cfd_x(p, mu, dxmu);
    err |= cfd_y(p, mu, dymu);
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        Fx[n] = -rho[n] * dxmu[n] + CS2 * dxr[n];
        Fy[n] = -rho[n] * dymu[n] + CS2 * dyr[n];
        if (mu_out)
            mu_out[n] = mu[n];
    }
    free(buf);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* MRT collision, Eq. 4                                                      */
/* ------------------------------------------------------------------------ */

/* The D2Q9 moment basis of the MRT model the paper cites (Lallemand and Luo):
 * rows rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy over the velocity order
 * of Sec. 2.  The paper does not print M; this is the standard basis its S =
 * diag(0, s_e, s_eps, 0, s_q, 0, s_q, s_v, s_v) is written for. */
static const double MRT_M[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

/* Inverse of a 9 x 9 matrix by Gauss-Jordan elimination with partial pivoting. */
static int invert9(const double a_in[9][9], double inv[9][9])
{
    double a[9][18];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 18; ++j)
            a[i][j] = j < 9 ? a_in[i][j] : (j - 9 == i ? 1.0 : 0.0);
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(a[r][c]) > fabs(a[piv][c]))
                piv = r;
        if (a[piv][c] == 0.0)
            return -1;
        for (int j = 0; j < 18; ++j) {
            double t = a[c][j];
            a[c][j] = a[piv][j];
            a[piv][j] = t;
        }
        double d = a[c][c];
        for (int j = 0; j < 18; ++j)
            a[c][j] /= d;
        for (int r = 0; r < 9; ++r)
            if (r != c) {
                double m = a[r][c];
                for (int j = 0; j < 18; ++j)
                    a[r][j] -= m * a[c][j];
            }
    }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j)
            inv[i][j] = a[i][9 + j];
    return 0;
}

/* Exported for the tests: M and its inverse. */
void orc_mrt_matrices(double *m_out, double *minv_out)
{
    double inv[9][9];
    invert9(MRT_M, inv);
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            m_out[9 * i + j] = MRT_M[i][j];
            minv_out[9 * i + j] = inv[i][j];
        }
}

/* Advance the post-streaming populations f (time level t0) by nsteps steps:
 * moments (Eq. 3), force stage, BGK collision with exact-difference forcing
 * (Eqs. 1, 2, 5), then streaming f_i(x + e_i, t + 1) = f_i*(x, t) on the
 * periodic lattice.  Returns 0 or -1. */
int orc_run(const orc_params *p, double *f, int64_t t0, int64_t nsteps)
{
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    double *buf = (double *)malloc(sizeof(double) * (5 * N + 9 * N));
    if (!buf)
        return -1;
    double *rho = buf, *ux = buf + N, *uy = buf + 2 * N, *Fx = buf + 3 * N,
           *Fy = buf + 4 * N, *fs = buf + 5 * N;
    int err = 0;
    double minv[9][9];
    if (p->mrt && invert9(MRT_M, minv))
        err = 1;
    for (int64_t s = 0; s < nsteps && !err; ++s) {
        int64_t t = t0 + s;
        moments(p, f, rho, ux, uy);
        err |= orc_force_stage(p, t, rho, NULL, Fx, Fy);
        /* collision: the right-hand side of Eq. 1 (BGK) or Eq. 4 (MRT,
         * f* = f - M^-1 S M (f - f^eq) + F_i) */
#pragma omp parallel for schedule(static)
        for (size_t n = 0; n < N; ++n) {
            double Fi[9];
            orc_forcing_terms(rho[n], ux[n], uy[n], Fx[n], Fy[n], Fi);
            if (!p->mrt) {
                for (int i = 0; i < 9; ++i) {
                    double fi = f[i * N + n];
                    fs[i * N + n] = fi - (fi - feq(i, rho[n], ux[n], uy[n])) / p->tau + Fi[i];
                }
                continue;
            }
            double dev[9], m[9];
            for (int i = 0; i < 9; ++i)
                dev[i] = f[i * N + n] - feq(i, rho[n], ux[n], uy[n]);
            for (int r = 0; r < 9; ++r) {
                m[r] = 0.0;
                for (int i = 0; i < 9; ++i)
                    m[r] += MRT_M[r][i] * dev[i];
                m[r] *= p->s[r];
            }
            for (int i = 0; i < 9; ++i) {
                double d = 0.0;
                for (int r = 0; r < 9; ++r)
                    d += minv[i][r] * m[r];
                fs[i * N + n] = f[i * N + n] - d + Fi[i];
            }
        }
        /* streaming, Eq. 1 left-hand side, periodic in x; in y periodic, or with
         * walls halfway bounce-back: a population that would leave the fluid
         * through a wall returns to its node in the opposite direction.  A wall
         * moving along x at U (a moving reference frame, Sec. 5.5) adds the
         * momentum of Ladd's moving-wall rule,
         *   f_opp(i)(x, t+1) = f*_i(x, t) - 2 w_i rho(x, t) (e_i . U) / c_s^2,
         * with rho the node's own density: mass is conserved, since the two
         * diagonals it changes cancel. */
        /* every destination is written by exactly one source, so the rows can
         * be shared among threads */
        for (int i = 0; i < 9; ++i)
#pragma omp parallel for schedule(static)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int xd = (x + EX[i] + nx) % nx, yd = y + EY[i];
                    double v = fs[i * N + (size_t)y * nx + x];
                    if (!p->walls_y) {
                        yd = (yd + ny) % ny;
                    } else if (yd < 0 || yd >= ny) {
                        double U = p->wall_ux[yd < 0 ? 0 : 1];
                        size_t n = (size_t)y * nx + x;
                        f[OPP[i] * N + n] = v - 2.0 * WQ[i] * rho[n] * EX[i] * U / CS2;
                        continue;
                    }
                    f[i * N + (size_t)yd * nx + xd] = v;
                }
    }
    free(buf);
    return err ? -1 : 0;
}

/* Macroscopic outputs of the state f at time level t:
 *   rho (Eq. 3), v = u + F/(2 rho) (Sec. 2, after Eq. 5), mu-hat (Eq. 33),
 *   and the force F of Eq. 12.  Any output but rho may be NULL. */
int orc_macro(const orc_params *p, const double *f, int64_t t, double *rho, double *vx,
              double *vy, double *mu, double *Fx_out, double *Fy_out)
{
    size_t N = (size_t)p->nx * p->ny;
    double *buf = (double *)malloc(sizeof(double) * 4 * N);
    if (!buf)
        return -1;
    double *ux = buf, *uy = buf + N, *Fx = buf + 2 * N, *Fy = buf + 3 * N;
    moments(p, f, rho, ux, uy);
    int err = orc_force_stage(p, t, rho, mu, Fx, Fy);
    for (size_t n = 0; n < N; ++n) {
        if (vx)
            vx[n] = ux[n] + Fx[n] / (2.0 * rho[n]);
        if (vy)
            vy[n] = uy[n] + Fy[n] / (2.0 * rho[n]);
        if (Fx_out)
            Fx_out[n] = Fx[n];
        if (Fy_out)
            Fy_out[n] = Fy[n];
    }
    free(buf);
    return err;
}
