// kernels_lbm.cu -- lattice kernels: fused collide-stream (Eqs. 1-5),
// equilibrium initialisation, moments, output velocity and diagnostics.
//
// Populations are structure-of-arrays, f[i*plane + y*nx + x], i in the velocity
// order of Sec. 2.  TF is the storage and arithmetic type of the populations:
// double (FP64 path) or float (mixed path).  The density and force fields are
// always FP64.
#include <cfloat>
#include <climits>

#include "cplbm_internal.cuh"
#include "lattice.cuh"

namespace cplbm {
namespace {

// D2Q9 velocity set and weights (Sec. 2).  Called with compile-time i inside
// fully unrolled loops, so they fold to constants.
__host__ __device__ __forceinline__ constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
template <typename T>
__host__ __device__ __forceinline__ constexpr T wq(int i) {
    return i == 0 ? T(4.0 / 9.0) : (i < 5 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}


template <typename T>
__device__ __forceinline__ T sum9(const T f[9]) {
    return ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
}

// Second-order equilibrium of Eq. 2 with c_s^2 = 1/3:
//   f_i^eq = w_i rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u).
template <typename T>
__device__ __forceinline__ T feq(int i, T rho, T ux, T uy, T uu) {
    const T eu = T(ex(i)) * ux + T(ey(i)) * uy;
    return wq<T>(i) * rho * (T(1) + T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
}

__device__ __forceinline__ void raise_flag(DevState* st, unsigned bits, int64_t t) {
    atomicOr(&st->flag, bits);
    atomicMin(&st->failed_t, (unsigned long long)t);
}

// ---------------------------------------------------------------------------
// Pass 1, FP64: fused collide + stream (pull from a shared-memory tile).
// A block owns a BX x BY tile of destination nodes.  It first collides the
// tile plus a one-node periodic halo (post-collision values to shared memory),
// then every destination node gathers f_i*(x - e_i) from shared memory, writes
// its nine populations once (coalesced, aligned) and its new density.
// ---------------------------------------------------------------------------
template <typename TF, int BX, int BY, bool MRT, bool WALLS>
__global__ void __launch_bounds__(BX* BY)
    k_collide_stream(const TF* __restrict__ fin, TF* __restrict__ fout,
                     const double* __restrict__ Fx, const double* __restrict__ Fy,
                     double* __restrict__ rho_out, int nx, int ny, size_t plane, TF omega,
                     TF se, TF seps, TF sq, TF uwb6, TF uwt6,
                     DevState* __restrict__ st) {
    constexpr int HX = BX + 2, HY = BY + 2, HN = HX * HY;
    __shared__ TF sf[9][HN];
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int gx0 = blockIdx.x * BX - 1, gy0 = blockIdx.y * BY - 1;
    bool ok = true;
    for (int k = tid; k < HN; k += BX * BY) {
        const int ly = k / HX, lx = k - ly * HX;
        const int gx = wrap_near(gx0 + lx, nx), gy = wrap_near(gy0 + ly, ny);
        const size_t n = (size_t)gy * nx + gx;
        TF f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fin[i * plane + n];
        if constexpr (MRT)
            ok &= collide_mrt<TF>(f, (TF)Fx[n], (TF)Fy[n], omega, (TF)FLT_MAX, se, seps, sq);
        else
            ok &= collide_pairs<TF>(f, (TF)Fx[n], (TF)Fy[n], omega, (TF)FLT_MAX);
#pragma unroll
        for (int i = 0; i < 9; ++i) sf[i][k] = f[i];
    }
    __syncthreads();
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x < nx && y < ny) {
        const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
        const size_t n = (size_t)y * nx + x;
        TF g[9];
        // the node's density, for the momentum a moving wall gives
        TF rw = TF(0);
        if (WALLS && (y == 0 || y == ny - 1)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) rw += sf[i][ly * HX + lx];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ys = y - q_ey(i);
            // halfway bounce-back at walls: the node's own opposite population,
            // plus e_x rho U / 6 on the diagonals from a wall moving at U (Ladd)
            if (WALLS && (ys < 0 || ys >= ny))
                g[i] = sf[q_opp(i)][ly * HX + lx] + TF(q_ex(i)) * rw * (ys < 0 ? uwb6 : uwt6);
            else
                g[i] = sf[i][(ly - q_ey(i)) * HX + (lx - q_ex(i))];
            fout[i * plane + n] = g[i];
        }
        rho_out[n] = (double)sum9(g);
    }
    if (!ok) raise_flag(st, FLAG_RHO, st->t);
}

// f_i = f_i^eq(rho, u) (Eq. 2) in FP64, stored as TF; rho_out = sum of the
// stored populations (the density every later pass sees).
template <typename TF>
__global__ void k_init_feq(const double* __restrict__ rho, const double* __restrict__ ux,
                           const double* __restrict__ uy, TF* __restrict__ f,
                           double* __restrict__ rho_out, size_t N, size_t plane) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const double r = rho[n];
        const double u = ux ? ux[n] : 0.0, v = uy ? uy[n] : 0.0;
        const double uu = u * u + v * v;
        TF g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            g[i] = (TF)feq<double>(i, r, u, v, uu);
            f[i * plane + n] = g[i];
        }
        rho_out[n] = (double)sum9(g);
    }
}

template <typename TF>
__global__ void k_rho_from_f(const TF* __restrict__ f, double* __restrict__ rho, size_t N,
                             size_t plane) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        TF g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = f[i * plane + n];
        rho[n] = (double)sum9(g);
    }
}

// Output velocity v = u + F/(2 rho) (Sec. 2, after Eq. 5), in FP64.
template <typename TF>
__device__ __forceinline__ void node_velocity(const TF* __restrict__ f, size_t plane, size_t n,
                                              double Fx, double Fy, double& rho, double& vx,
                                              double& vy) {
    double g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = (double)f[i * plane + n];
    rho = sum9(g);
    const double jx = (g[1] + g[5] + g[8]) - (g[3] + g[6] + g[7]);
    const double jy = (g[2] + g[5] + g[6]) - (g[4] + g[7] + g[8]);
    vx = (jx + 0.5 * Fx) / rho;
    vy = (jy + 0.5 * Fy) / rho;
}

template <typename TF>
__global__ void k_macro(const TF* __restrict__ f, const double* __restrict__ Fx,
                        const double* __restrict__ Fy, double* __restrict__ vx,
                        double* __restrict__ vy, size_t N, size_t plane) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        double r, u, v;
        node_velocity(f, plane, n, Fx[n], Fy[n], r, u, v);
        if (vx) vx[n] = u;
        if (vy) vy[n] = v;
    }
}

// Diagnostics, two deterministic stages: per-block partials, then one block.
constexpr int kDiagThreads = 256;

template <typename TF>
__global__ void __launch_bounds__(kDiagThreads)
    k_diag_partial(const TF* __restrict__ f, const double* __restrict__ rho,
                   const double* __restrict__ Fx, const double* __restrict__ Fy, size_t N,
                   size_t plane, double* __restrict__ partials) {
    double s = 0.0, vmax = 0.0, rmin = DBL_MAX, rmax = -DBL_MAX;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        double r, u, v;
        node_velocity(f, plane, n, Fx[n], Fy[n], r, u, v);
        const double rf = rho[n];
        s += rf;
        vmax = fmax(vmax, sqrt(u * u + v * v));
        rmin = fmin(rmin, rf);
        rmax = fmax(rmax, rf);
    }
    __shared__ double sh[4][kDiagThreads];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = vmax;
    sh[2][threadIdx.x] = rmin;
    sh[3][threadIdx.x] = rmax;
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) partials[4 * blockIdx.x + q] = sh[q][0];
    }
}

__global__ void __launch_bounds__(kDiagThreads)
    k_diag_final(const double* __restrict__ partials, int nparts, DevState* __restrict__ st) {
    double s = 0.0, vmax = 0.0, rmin = DBL_MAX, rmax = -DBL_MAX;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        s += partials[4 * b];
        vmax = fmax(vmax, partials[4 * b + 1]);
        rmin = fmin(rmin, partials[4 * b + 2]);
        rmax = fmax(rmax, partials[4 * b + 3]);
    }
    __shared__ double sh[4][kDiagThreads];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = vmax;
    sh[2][threadIdx.x] = rmin;
    sh[3][threadIdx.x] = rmax;
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) st->diag[q] = sh[q][0];
    }
}

template <typename TF>
__global__ void k_f_to_double(const TF* __restrict__ f, double* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)f[i];
}

template <typename TF>
__global__ void k_f_from_double(const double* __restrict__ in, TF* __restrict__ f, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        f[i] = (TF)in[i];
}

inline unsigned grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 65535 * 16 ? (b ? b : 1) : 65535 * 16);
}

}  // namespace

// Tile of the collide-stream pass: 32 x 8 destination nodes per block.
constexpr int kCsBX = 32, kCsBY = 16;

template <typename TF>
cudaError_t launch_collide_stream(const TF* fin, TF* fout, const double* Fx, const double* Fy,
                                  double* rho_out, int nx, int ny, size_t plane, double omega,
                                  const MrtRates* mrt, DevState* st, cudaStream_t s,
                                  const Walls& walls) {
    const TF ub = (TF)(walls.u[0] / 6.0), ut = (TF)(walls.u[1] / 6.0);
    dim3 block(kCsBX, kCsBY);
    dim3 grid((nx + kCsBX - 1) / kCsBX, (ny + kCsBY - 1) / kCsBY);
    const TF se = mrt ? (TF)mrt->se : TF(0), seps = mrt ? (TF)mrt->seps : TF(0),
             sq = mrt ? (TF)mrt->sq : TF(0);
#define CPLBM_CS(M, W)                                                                    \
    k_collide_stream<TF, kCsBX, kCsBY, M, W><<<grid, block, 0, s>>>(                      \
        fin, fout, Fx, Fy, rho_out, nx, ny, plane, (TF)omega, se, seps, sq, ub, ut, st)
    if (mrt && walls.on)
        CPLBM_CS(true, true);
    else if (mrt)
        CPLBM_CS(true, false);
    else if (walls.on)
        CPLBM_CS(false, true);
    else
        CPLBM_CS(false, false);
#undef CPLBM_CS
    return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_init_feq(const double* rho, const double* ux, const double* uy, TF* f,
                            double* rho_out, int nx, int ny, size_t plane, cudaStream_t s) {
    size_t N = (size_t)nx * ny;
    k_init_feq<TF><<<grid_for(N, 256), 256, 0, s>>>(rho, ux, uy, f, rho_out, N, plane);
    return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_rho_from_f(const TF* f, double* rho, int nx, int ny, size_t plane,
                              cudaStream_t s) {
    size_t N = (size_t)nx * ny;
    k_rho_from_f<TF><<<grid_for(N, 256), 256, 0, s>>>(f, rho, N, plane);
    return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_macro(const TF* f, const double* Fx, const double* Fy, double* vx,
                         double* vy, int nx, int ny, size_t plane, cudaStream_t s) {
    size_t N = (size_t)nx * ny;
    k_macro<TF><<<grid_for(N, 256), 256, 0, s>>>(f, Fx, Fy, vx, vy, N, plane);
    return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_diag(const TF* f, const double* rho, const double* Fx, const double* Fy,
                        int nx, int ny, size_t plane, double* partials, int nparts,
                        DevState* st, cudaStream_t s) {
    size_t N = (size_t)nx * ny;
    k_diag_partial<TF><<<nparts, kDiagThreads, 0, s>>>(f, rho, Fx, Fy, N, plane, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final<<<1, kDiagThreads, 0, s>>>(partials, nparts, st);
    return cudaGetLastError();
}

cudaError_t launch_diag_final(const double* partials, int nparts, DevState* st, cudaStream_t s) {
    k_diag_final<<<1, kDiagThreads, 0, s>>>(partials, nparts, st);
    return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_f_to_double(const TF* f, double* out, size_t n, cudaStream_t s) {
    k_f_to_double<TF><<<grid_for(n, 256), 256, 0, s>>>(f, out, n);
    return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_f_from_double(const double* in, TF* f, size_t n, cudaStream_t s) {
    k_f_from_double<TF><<<grid_for(n, 256), 256, 0, s>>>(in, f, n);
    return cudaGetLastError();
}

#define CPLBM_INST(TF)                                                                       \
    template cudaError_t launch_collide_stream<TF>(const TF*, TF*, const double*,            \
                                                   const double*, double*, int, int, size_t, \
                                                   double, const MrtRates*, DevState*,       \
                                                   cudaStream_t, const Walls&);              \
    template cudaError_t launch_init_feq<TF>(const double*, const double*, const double*,    \
                                             TF*, double*, int, int, size_t, cudaStream_t);  \
    template cudaError_t launch_rho_from_f<TF>(const TF*, double*, int, int, size_t,         \
                                               cudaStream_t);                                \
    template cudaError_t launch_macro<TF>(const TF*, const double*, const double*, double*,  \
                                          double*, int, int, size_t, cudaStream_t);          \
    template cudaError_t launch_diag<TF>(const TF*, const double*, const double*,            \
                                         const double*, int, int, size_t, double*, int,      \
                                         DevState*, cudaStream_t);                           \
    template cudaError_t launch_f_to_double<TF>(const TF*, double*, size_t, cudaStream_t);   \
    template cudaError_t launch_f_from_double<TF>(const double*, TF*, size_t, cudaStream_t);

CPLBM_INST(double)
CPLBM_INST(float)
#undef CPLBM_INST

}  // namespace cplbm
