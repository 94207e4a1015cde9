// kernels_cfd.cu -- compact finite-difference line solves (Eqs. 37-39) and
// the fused force stage: chemical potential (Eqs. 21, 33, Sec. 5.6 limit) and
// nonideal force (Eq. 12).
//
// Solver.  On a periodic line the compact scheme is the circulant system
//   A d = B u,  (A d)_i = alpha d_{i-1} + d_i + alpha d_{i+1},
//   (B u)_i = a/2 (u_{i+1} - u_{i-1}) + b/4 (u_{i+2} - u_{i-2}).
// A factors into two first-order recursions (see CfdCoef):
//   forward   w_i = r_i - lam w_{i-1}         (1 + lam S^-1) w = r
//   backward  z_i = w_i - lam z_{i+1}         (1 + lam S)    z = w
// with r = (lam/alpha) B u and d = z.  Because |lam| < 1 (0.382 for alpha=1/3,
// 0.268 for alpha=1/4), the weight of a value q positions away decays as
// lam^q; a recursion started `warm` positions before the first output is exact
// to FP64 rounding, whatever the line length (positions are taken mod n, so
// short lines simply wrap).  This replaces the serial Thomas sweep of the
// paper (Sec. 4.3) by independent line segments: one thread sweeps one segment
// [s, e) of one line.  The forward sweep stores w for [s, e) in the output
// arrays, and sums the backward recursion's starting value over [e, e+warm)
// on the fly, so no scratch memory is needed; the backward sweep then reads w
// back and writes the result through a fused epilogue.
//
// Second derivative ("applying CFM twice", Sec. 4.3): D(D u) with D = A^-1 B.
// All these operators are circulant and commute, so D D u = F_b F_b F_f F_f (B B u)
// with F_f, F_b the forward/backward recursions; one sweep carries both.
#include <cmath>

#include "cplbm_internal.cuh"

namespace cplbm {

CfdCoef make_cfd_coef(int fd_order) {
    const double alpha = fd_order == 6 ? 1.0 / 3.0 : 0.25;
    const double a = 2.0 / 3.0 * (alpha + 2.0);  // Eq. 38
    const double b = (4.0 * alpha - 1.0) / 3.0;  // Eq. 38
    const double lam = (1.0 - std::sqrt(1.0 - 4.0 * alpha * alpha)) / (2.0 * alpha);
    CfdCoef c;
    c.c1 = lam / alpha * a / 2.0;
    c.c2 = lam / alpha * b / 4.0;
    c.lam = lam;
    // smallest q with (q+1) lam^q < 1e-18 (the double recursion's tail weight)
    int q = 1;
    while ((q + 1) * std::pow(lam, q) > 1e-18) ++q;
    c.warm = q;
    c.sixth = fd_order == 6 ? 1 : 0;
    return c;
}

int default_segment(int line_len, int n_lines) {
    // Enough independent segments to fill the GPU (about 38k threads), segments
    // no shorter than 32 (the warm-up is amortised over the segment).
    const double want = 38912.0;
    double seg = (double)line_len * (double)n_lines / want;
    int s = (int)seg;
    if (s < 32) s = 32;
    if (s > 256) s = 256;
    if (s > line_len) s = line_len;
    return s;
}

namespace {

__device__ __forceinline__ int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
__device__ __forceinline__ int nexti(int v, int n) { return v + 1 == n ? 0 : v + 1; }
__device__ __forceinline__ int previ(int v, int n) { return v == 0 ? n - 1 : v - 1; }

// One segment [s, e) of one periodic line of length n.  Element at line
// position p lives at global offset off0 + p*ps.  SIXTH: the +-2 neighbours
// enter the right-hand side.  SECOND: also produce D(D u).
// t1 / t2 receive the forward states for [s, e) and are read back; epi(o, d1,
// d2) is called once per position with the final values.
template <bool SIXTH, bool SECOND, class Epi>
__device__ __forceinline__ void line_sweep(const double* __restrict__ u, double* t1, double* t2,
                                           size_t off0, ptrdiff_t ps, int n, int s, int e,
                                           const CfdCoef& c, Epi& epi) {
    const double lam = c.lam, c1 = c.c1, c2 = c.c2;
    const int W = c.warm;
    constexpr int L = SECOND ? 2 : 0;  // lag of the processed position behind the b1 front

    // u window u_{j-2..j+2} for b1_j
    double um2 = 0.0, um1, u0, up1, up2;
    const int jstart = s - W - L;
    int iu = wrapi(jstart - 2, n);
    um1 = __ldg(u + off0 + (ptrdiff_t)iu * ps);
    iu = nexti(iu, n);
    u0 = __ldg(u + off0 + (ptrdiff_t)iu * ps);
    iu = nexti(iu, n);
    up1 = __ldg(u + off0 + (ptrdiff_t)iu * ps);
    iu = nexti(iu, n);
    up2 = __ldg(u + off0 + (ptrdiff_t)iu * ps);
    iu = nexti(iu, n);

    double b1m2 = 0.0, b1m1 = 0.0, b10 = 0.0, b1p1 = 0.0, b1p2 = 0.0;
    double w1 = 0.0, v = 0.0, w2 = 0.0;

    // advance the b1 front by one position and return b1 at the processed position
    auto advance = [&](double& b1c, double& b2c) {
        um2 = um1;
        um1 = u0;
        u0 = up1;
        up1 = up2;
        up2 = __ldg(u + off0 + (ptrdiff_t)iu * ps);
        iu = nexti(iu, n);
        double b1 = c1 * (up1 - um1);
        if (SIXTH) b1 = fma(c2, up2 - um2, b1);
        if (SECOND) {
            b1m2 = b1m1;
            b1m1 = b10;
            b10 = b1p1;
            b1p1 = b1p2;
            b1p2 = b1;
            double b2 = c1 * (b1p1 - b1m1);
            if (SIXTH) b2 = fma(c2, b1p2 - b1m2, b2);
            b1c = b10;
            b2c = b2;
        } else {
            b1c = b1;
            b2c = 0.0;
        }
    };
    // (um1, u0, up1, up2) = u_{jstart-2 .. jstart+1}; iu -> jstart+2, so the
    // first advance() yields b1 at jstart.
    double b1c, b2c;
    // prime the b1 window (SECOND needs b1 at p-2..p+2 before position p)
    for (int k = 0; k < 2 * L; ++k) advance(b1c, b2c);
    // warm-up: positions s-W .. s-1
    for (int k = 0; k < W; ++k) {
        advance(b1c, b2c);
        w1 = b1c - lam * w1;
        if (SECOND) {
            v = b2c - lam * v;
            w2 = v - lam * w2;
        }
    }
    // owned positions s .. e-1: store the forward states
    int io = wrapi(s, n);
    for (int p = s; p < e; ++p) {
        advance(b1c, b2c);
        w1 = b1c - lam * w1;
        const size_t o = off0 + (ptrdiff_t)io * ps;
        t1[o] = w1;
        if (SECOND) {
            v = b2c - lam * v;
            w2 = v - lam * w2;
            t2[o] = w2;
        }
        io = nexti(io, n);
    }
    // tail e .. e+W-1: starting values of the backward recursions
    //   z1_e = sum_q (-lam)^q w1_{e+q},  y_e = sum_q (-lam)^q w2_{e+q},
    //   z2_e = sum_q (q+1)(-lam)^q w2_{e+q}
    double acc1 = 0.0, accy = 0.0, accz = 0.0, pw = 1.0;
    for (int q = 0; q < W; ++q) {
        advance(b1c, b2c);
        w1 = b1c - lam * w1;
        acc1 = fma(pw, w1, acc1);
        if (SECOND) {
            v = b2c - lam * v;
            w2 = v - lam * w2;
            accy = fma(pw, w2, accy);
            accz = fma((double)(q + 1) * pw, w2, accz);
        }
        pw *= -lam;
    }
    // backward sweep over e-1 .. s
    double z1 = acc1, y = accy, z2 = accz;
    io = wrapi(e - 1, n);
    for (int p = e - 1; p >= s; --p) {
        const size_t o = off0 + (ptrdiff_t)io * ps;
        z1 = t1[o] - lam * z1;
        if (SECOND) {
            y = t2[o] - lam * y;
            z2 = y - lam * z2;
        }
        epi(o, z1, z2);
        io = previ(io, n);
    }
}

struct EpiStore {
    double* d1;
    double* d2;
    __device__ __forceinline__ void operator()(size_t o, double a, double b) {
        d1[o] = a;
        if (d2) d2[o] = b;
    }
};

// Pass 3 epilogue: d_y rho, then mu-hat = k^2 mu0(rho) - kappa (d_xx + d_yy) rho
// (Eqs. 21, 33) with the upper limit of Sec. 5.6.
struct EpiMu {
    double* dyr;
    double* mu;
    const double* __restrict__ rho;
    const double* __restrict__ dxx;
    PhysParams p;
    bool capped;
    int64_t t;
    bool bad;
    __device__ __forceinline__ void operator()(size_t o, double d1, double d2) {
        dyr[o] = d1;
        const double r = rho[o];
        const double eta = 0.25 * p.b * r;
        const double om = 1.0 - eta;
        // Carnahan-Starling chemical potential, Eq. 21 without the gradient term
        const double mu0 = p.R * p.T * ((3.0 - eta) / (om * om * om) + log(r) + 1.0) -
                           2.0 * p.a * r;
        double m = p.k2 * mu0 - p.kappa * (dxx[o] + d2);
        if (capped) m = fmin(m, p.mu_cap);
        bad |= !(r > 0.0 && eta < 1.0 && fabs(m) < 1e300);
        mu[o] = m;
    }
};

// Passes 4/5 epilogue: F = -rho d(mu-hat) + c_s^2 d(rho) (Eq. 12).
struct EpiForce {
    double* F;
    const double* __restrict__ rho;
    const double* __restrict__ dr;
    __device__ __forceinline__ void operator()(size_t o, double dmu, double) {
        F[o] = fma(-rho[o], dmu, dr[o] * (1.0 / 3.0));
    }
};

// Thread -> (line, segment).  Consecutive threads take consecutive lines, so
// for y-lines (line stride 1) every load and store of a warp is coalesced.
struct LineMap {
    int n;           // line length
    int nlines;
    ptrdiff_t ps;    // stride along a line
    ptrdiff_t ls;    // stride between lines
    int seg, nseg;
};

template <bool SIXTH, bool SECOND, class Epi>
__device__ __forceinline__ bool run_line(const double* __restrict__ u, double* t1, double* t2,
                                         const LineMap& m, const CfdCoef& c, Epi& epi) {
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)m.nlines * m.nseg) return false;
    const int line = (int)(gid % m.nlines), sg = (int)(gid / m.nlines);
    const int s = sg * m.seg;
    const int e = min(s + m.seg, m.n);
    line_sweep<SIXTH, SECOND>(u, t1, t2, (size_t)line * m.ls, m.ps, m.n, s, e, c, epi);
    return true;
}

template <bool SIXTH, bool SECOND>
__global__ void __launch_bounds__(128)
    k_cfd_plain(const double* __restrict__ u, double* d1, double* d2, LineMap m, CfdCoef c,
                DevState* st, int bump) {
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) st->t += 1;
    EpiStore epi{d1, d2};
    run_line<SIXTH, SECOND>(u, d1, d2, m, c, epi);
}

template <bool SIXTH>
__global__ void __launch_bounds__(128)
    k_cfd_mu(const double* __restrict__ rho, const double* __restrict__ dxx, double* dyr,
             double* mu, LineMap m, CfdCoef c, PhysParams p, DevState* st) {
    const int64_t t = st->t;
    EpiMu epi{dyr, mu, rho, dxx, p, t < p.cap_steps, t, false};
    run_line<SIXTH, true>(rho, dyr, mu, m, c, epi);
    if (epi.bad) {
        atomicOr(&st->flag, FLAG_EOS);
        atomicMin(&st->failed_t, (unsigned long long)t);
    }
}

template <bool SIXTH>
__global__ void __launch_bounds__(128)
    k_cfd_force(const double* __restrict__ mu, const double* __restrict__ rho,
                const double* __restrict__ dr, double* F, LineMap m, CfdCoef c) {
    EpiForce epi{F, rho, dr};
    run_line<SIXTH, false>(mu, F, nullptr, m, c, epi);
}

LineMap make_map(int nx, int ny, int axis, int seg) {
    LineMap m;
    if (axis == 0) {
        m.n = nx;
        m.nlines = ny;
        m.ps = 1;
        m.ls = nx;
    } else {
        m.n = ny;
        m.nlines = nx;
        m.ps = nx;
        m.ls = 1;
    }
    m.seg = seg > 0 ? (seg < m.n ? seg : m.n) : default_segment(m.n, m.nlines);
    m.nseg = (m.n + m.seg - 1) / m.seg;
    return m;
}

constexpr int kThreads = 128;
inline unsigned blocks_for(const LineMap& m) {
    long t = (long)m.nlines * m.nseg;
    return (unsigned)((t + kThreads - 1) / kThreads);
}

}  // namespace

static cudaError_t plain(const double* u, double* d1, double* d2, int nx, int ny, int axis,
                         int seg, const CfdCoef& c, DevState* st, int bump, cudaStream_t s) {
    LineMap m = make_map(nx, ny, axis, seg);
    const unsigned g = blocks_for(m);
    if (c.sixth) {
        if (d2)
            k_cfd_plain<true, true><<<g, kThreads, 0, s>>>(u, d1, d2, m, c, st, bump);
        else
            k_cfd_plain<true, false><<<g, kThreads, 0, s>>>(u, d1, d2, m, c, st, bump);
    } else {
        if (d2)
            k_cfd_plain<false, true><<<g, kThreads, 0, s>>>(u, d1, d2, m, c, st, bump);
        else
            k_cfd_plain<false, false><<<g, kThreads, 0, s>>>(u, d1, d2, m, c, st, bump);
    }
    return cudaGetLastError();
}

cudaError_t launch_cfd_plain(const double* u, double* d1, double* d2, int nx, int ny, int axis,
                             int seg, const CfdCoef& c, cudaStream_t s) {
    return plain(u, d1, d2, nx, ny, axis, seg, c, nullptr, 0, s);
}

cudaError_t launch_cfd_x_rho(const double* rho, double* dxr, double* dxx, int nx, int ny,
                             int seg, const CfdCoef& c, DevState* st, int bump,
                             cudaStream_t s) {
    return plain(rho, dxr, dxx, nx, ny, 0, seg, c, st, bump, s);
}

cudaError_t launch_cfd_y_rho_mu(const double* rho, const double* dxx, double* dyr, double* mu,
                                int nx, int ny, int seg, const CfdCoef& c,
                                const PhysParams& p, DevState* st, cudaStream_t s) {
    LineMap m = make_map(nx, ny, 1, seg);
    const unsigned g = blocks_for(m);
    if (c.sixth)
        k_cfd_mu<true><<<g, kThreads, 0, s>>>(rho, dxx, dyr, mu, m, c, p, st);
    else
        k_cfd_mu<false><<<g, kThreads, 0, s>>>(rho, dxx, dyr, mu, m, c, p, st);
    return cudaGetLastError();
}

static cudaError_t force(const double* mu, const double* rho, const double* dr, double* F,
                         int nx, int ny, int axis, int seg, const CfdCoef& c, cudaStream_t s) {
    LineMap m = make_map(nx, ny, axis, seg);
    const unsigned g = blocks_for(m);
    if (c.sixth)
        k_cfd_force<true><<<g, kThreads, 0, s>>>(mu, rho, dr, F, m, c);
    else
        k_cfd_force<false><<<g, kThreads, 0, s>>>(mu, rho, dr, F, m, c);
    return cudaGetLastError();
}

cudaError_t launch_cfd_x_force(const double* mu, const double* rho, const double* dxr,
                               double* Fx, int nx, int ny, int seg, const CfdCoef& c,
                               cudaStream_t s) {
    return force(mu, rho, dxr, Fx, nx, ny, 0, seg, c, s);
}

cudaError_t launch_cfd_y_force(const double* mu, const double* rho, const double* dyr,
                               double* Fy, int nx, int ny, int seg, const CfdCoef& c,
                               cudaStream_t s) {
    return force(mu, rho, dyr, Fy, nx, ny, 1, seg, c, s);
}

}  // namespace cplbm
