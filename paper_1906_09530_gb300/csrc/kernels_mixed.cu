// kernels_mixed.cu -- lattice kernels of the mixed-precision path: FP32
// populations and collision, the density kept as a double-float pair; its line
// solves are in kernels_lines.cu (double-float first derivatives of the density,
// FP32 second derivatives, chemical potential and force).
//
// Why this split (GB300 runs FP64 at 1/64 of the FP32 rate, so FP64 arithmetic
// in the line solves would bound the whole step):
//   * The density is the sum of nine FP32 populations; it is kept exactly, as an
//     unevaluated sum hi + lo of two floats ("double-float", DF).
//   * d rho enters the force (Eq. 12).  Near an interface a compact-FD line
//     solve mixes liquid-scale values into gas-side derivatives with weight
//     lam^d; FP32 rounding there (6e-8 of rho_l) would be an error of relative
//     size ~6e-8 rho_l / rho_g in the gas gradient, i.e. an inconsistent force
//     that shifts the coexistence density.  The solve is therefore carried in DF
//     (about 2^-44 relative to the line's values) and only the result is rounded
//     to FP32, which is relative to the derivative's own magnitude.
//   * d_xx rho, d_yy rho enter mu-hat multiplied by kappa; mu0 and mu-hat are
//     O(T ln rho); the force is rounded relative to itself.  FP32 errors in these
//     move mu by ~1e-7 of its size, i.e. relative density shifts ~1e-6, far below
//     the 1e-3 coexistence tolerance.
// FP32 rounding of all DF operations is forced with __fadd_rn/__fmul_rn so the
// compiler cannot contract them into fused multiply-adds.
#include <cfloat>
#include <cmath>

#include "cplbm_internal.cuh"
#include "df.cuh"
#include "eos.cuh"
#include "lattice.cuh"

namespace cplbm {

namespace {


// D2Q9 (Sec. 2)
__host__ __device__ __forceinline__ constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}


__device__ __forceinline__ void raise_flag(DevState* st, unsigned bits, int64_t t) {
    atomicOr(&st->flag, bits);
    atomicMin(&st->failed_t, (unsigned long long)t);
}

// ---------------------------------------------------------------------------
// Pass 1, mixed, sliding-window form: one warp owns 30 destination columns
// (lanes 1..30; lanes 0 and 31 collide the one-column halo) and walks down a
// strip of rows.  The post-collision populations of rows y-1, y and y+1 stay in
// registers; the pull f_i(x, y) = f_i*(x - e_i) takes the row from those three
// and the column from the lane itself or a neighbour lane (warp shuffle).  The
// loads of the next row are issued before the current row is finished.  No
// shared memory, no block barrier.
// ---------------------------------------------------------------------------
constexpr int kSwWarps = 4;  // warps per block

// Halfway bounce-back at a wall, by the ordinary pull: the populations that the
// pull takes from the solid row (H, the row beyond the wall) are replaced by the
// wall row's own populations moving into the wall, reversed, so each node gets
// its own reflected population.  A wall moving along x at U adds e_x rho U / 6
// on the diagonals (Ladd), rho the node's density.  Diagonals are placed one
// lane over, where the pull takes them from the neighbour lane.  Warp-uniform.
template <bool BOTTOM>
__device__ __forceinline__ void reflect_into(float (&H)[9], const float (&B)[9], float uw6) {
    float r = B[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) r = __fadd_rn(r, B[i]);
    const float c = __fmul_rn(r, uw6);
    if (BOTTOM) {  // H is row -1: directions 2, 5, 6 come from it
        H[2] = B[4];
        H[5] = __shfl_down_sync(0xffffffffu, __fadd_rn(B[7], c), 1);
        H[6] = __shfl_up_sync(0xffffffffu, __fsub_rn(B[8], c), 1);
    } else {  // H is row ny: directions 4, 7, 8 come from it
        H[4] = B[2];
        H[7] = __shfl_up_sync(0xffffffffu, __fsub_rn(B[5], c), 1);
        H[8] = __shfl_down_sync(0xffffffffu, __fadd_rn(B[6], c), 1);
    }
}

// WALLS: the bounce-back rows are compiled only into the walled variant, so
// the periodic kernel keeps its register count.
template <bool MRT, bool WALLS>
__device__ __forceinline__ void cs_mixed_body(const CsArgs& a, int wid) {
    const float* __restrict__ fin = a.fin;
    float* __restrict__ fout = a.fout;
    const float* __restrict__ Fx = a.Fx;
    const float* __restrict__ Fy = a.Fy;
    const int nx = a.nx, ny = a.ny;
    const size_t plane = a.plane;
    const float omega = a.omega;
    const int lane = threadIdx.x & 31;
    if (wid >= a.nstrips * a.nseg) return;  // uniform per warp
    const int strip = wid % a.nstrips, seg = wid / a.nstrips;
    const int x0 = strip * 30;
    const int gx = wrap_near(x0 - 1 + lane, nx);
    const int xo = x0 + lane - 1;
    const bool writer = lane >= 1 && lane <= 30 && xo < nx;
    const int y0 = seg * a.rows;
    const int y1 = min(y0 + a.rows, ny);
    bool ok = true;

    float raw[11];
    auto fetch = [&](int yr) {
        const size_t n = (size_t)wrap_near(yr, ny) * nx + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) raw[i] = fin[i * plane + n];
        raw[9] = Fx[n];
        raw[10] = Fy[n];
    };
    auto collide_raw = [&](float out[9]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i] = raw[i];
        if constexpr (MRT)
            ok &= collide_mrt<float>(out, raw[9], raw[10], omega, FLT_MAX, a.se, a.seps, a.sq);
        else
            ok &= collide_pairs<float>(out, raw[9], raw[10], omega, FLT_MAX);
    };
    float A[9], B[9], C[9];
    fetch(y0 - 1);
    collide_raw(A);
    fetch(y0);
    collide_raw(B);
    fetch(y0 + 1);
    if (WALLS && y0 == 0) reflect_into<true>(A, B, a.uw6[0]);
    for (int y = y0; y < y1; ++y) {
        if (WALLS && y == ny - 1) {
            // row ny is solid: the pull takes only C[4], C[7], C[8] from it
            reflect_into<false>(C, B, a.uw6[1]);
        } else {
            collide_raw(C);  // row y+1
            if (y + 1 < y1 && !(WALLS && y + 2 == ny)) fetch(y + 2);
        }
        // gather row y: e = (ex, ey) comes from row y - ey, column x - ex
        float g[9];
        g[0] = B[0];
        g[1] = __shfl_up_sync(0xffffffffu, B[1], 1);
        g[2] = A[2];
        g[3] = __shfl_down_sync(0xffffffffu, B[3], 1);
        g[4] = C[4];
        g[5] = __shfl_up_sync(0xffffffffu, A[5], 1);
        g[6] = __shfl_down_sync(0xffffffffu, A[6], 1);
        g[7] = __shfl_down_sync(0xffffffffu, C[7], 1);
        g[8] = __shfl_up_sync(0xffffffffu, C[8], 1);
        if (writer) {
            const size_t n = (size_t)y * nx + xo;
#pragma unroll
            for (int i = 0; i < 9; ++i) fout[i * plane + n] = g[i];
            const df r = sum9_exact(g);
            a.rh[n] = r.hi;
            a.rl[n] = r.lo;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            A[i] = B[i];
            B[i] = C[i];
        }
    }
    if (!ok) raise_flag(a.st, FLAG_RHO, a.st->t);
}

template <bool MRT>
__global__ void __launch_bounds__(kSwWarps * 32) k_cs_mixed_sw(CsArgs a) {
    pdl_prologue();
    cs_mixed_body<MRT, false>(a, blockIdx.x * kSwWarps + (threadIdx.x >> 5));
}

// With walls: held to the periodic kernel's 48 registers (10 blocks of 4 warps
// per SM); unconstrained, the wall rows cost one more 8-register granule and
// a tenth of the occupancy.
template <bool MRT>
__global__ void __launch_bounds__(kSwWarps * 32, 10) k_cs_mixed_sw_walls(CsArgs a) {
    pdl_prologue();
    cs_mixed_body<MRT, true>(a, blockIdx.x * kSwWarps + (threadIdx.x >> 5));
}

// ---------------------------------------------------------------------------
// Pass 1, mixed, row-ring form (periodic grids, nx a multiple of 4 and at least
// kRingT): a block of kRingT threads owns the kRingW destination columns
// [x0, x0 + kRingW), x0 = kRingW s, and a segment of rows [y0, y1); thread t
// stands for column x0 - 4 + t (periodically).  The raw rows y0 - 1 .. y1 (nine
// populations and the two force components, 128 columns from the 16-byte-aligned
// column x0 - 4) stream into a ring of kRingD row slots in shared memory, kRingD
// - 1 rows ahead of use, as 16-byte asynchronous copies: 352 pieces a row, three
// per thread, each piece four columns of one plane (nx a multiple of 4 puts every
// periodic seam on a piece boundary).  Every thread collides its column of the
// next row from the ring into a ring of post-collision rows; after a block
// barrier the threads of columns x0 .. x0 + kRingW - 1 gather row y from rows
// y - 1, y, y + 1 and columns x - 1, x, x + 1 and write it.  The collision and
// the gather are the sliding-window kernel's (same rounding), so the results are
// bit-identical; what changes is how many rows are in flight per thread and that
// no halo lane is wasted per warp.
// ---------------------------------------------------------------------------
constexpr int kRingT = 128, kRingW = kRingT - 8, kRingD = 5;
constexpr int kRingPieces = 11 * kRingT / 4;  // 16-byte pieces a row
constexpr int kRingPer = (kRingPieces + kRingT - 1) / kRingT;

__device__ __forceinline__ void ring_cp16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void ring_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void ring_wait_groups() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <bool MRT>
__global__ void __launch_bounds__(kRingT) k_cs_mixed_ring(CsArgs a) {
    pdl_prologue();
    __shared__ __align__(16) float raw[kRingD][11 * kRingT];
    // three post-collision rows: row r overwrites row r - 3, whose last reader
    // (the gather of row r - 2) finished before the barrier that precedes it
    __shared__ __align__(16) float post[3][9][kRingT];
    const int t = threadIdx.x;
    const int strip = blockIdx.x % a.nstrips, seg = blockIdx.x / a.nstrips;
    const int x0 = strip * kRingW, xa = x0 - 4;
    const int y0 = seg * a.rows, y1 = min(y0 + a.rows, a.ny);
    const int R = y1 - y0 + 2;  // rows y0 - 1 .. y1
    const int nx = a.nx, ny = a.ny;
    const size_t plane = a.plane;
    // this thread's pieces: plane, source column (wrapped), offset in a slot
    const float* src[kRingPer];
    int off[kRingPer];
#pragma unroll
    for (int j = 0; j < kRingPer; ++j) {
        const int k = t + j * kRingT;
        const int p = k < kRingPieces ? k / (kRingT / 4) : 0;
        const int c = k - p * (kRingT / 4);
        const float* base = p < 9 ? a.fin + (size_t)p * plane : (p == 9 ? a.Fx : a.Fy);
        src[j] = base + wrap_near(xa + 4 * c, nx);
        off[j] = k < kRingPieces ? p * kRingT + 4 * c : -1;
    }
    auto issue = [&](int r) {  // raw row y0 - 1 + r into slot r % kRingD
        const size_t row = (size_t)wrap_near(y0 - 1 + r, ny) * nx;
        float* slot = raw[r % kRingD];
#pragma unroll
        for (int j = 0; j < kRingPer; ++j)
            if (off[j] >= 0) ring_cp16(slot + off[j], src[j] + row);
    };
#pragma unroll
    for (int r = 0; r < kRingD; ++r) {
        if (r < R) issue(r);
        ring_commit();  // one group a row, empty past the end, so the count stays uniform
    }
    const int xo = xa + t;  // the column this thread writes (threads 4 .. kRingT - 5)
    const bool writer = t >= 4 && t < kRingT - 4 && xo < nx;
    bool ok = true;
    for (int r = 0; r < R; ++r) {
        if (r >= 1) {
            // slot (r - 1) % kRingD was read by every thread before the last barrier
            if (r - 1 + kRingD < R) issue(r - 1 + kRingD);
            ring_commit();
        }
        ring_wait_groups<kRingD - 1>();  // this thread's pieces of row r have landed
        __syncthreads();                 // and everyone's
        {
            float f[9];
            const float* w = raw[r % kRingD];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = w[i * kRingT + t];
            const float fx = w[9 * kRingT + t], fy = w[10 * kRingT + t];
            if constexpr (MRT)
                ok &= collide_mrt<float>(f, fx, fy, a.omega, FLT_MAX, a.se, a.seps, a.sq);
            else
                ok &= collide_pairs<float>(f, fx, fy, a.omega, FLT_MAX);
#pragma unroll
            for (int i = 0; i < 9; ++i) post[r % 3][i][t] = f[i];
        }
        __syncthreads();
        if (r >= 2 && writer) {
            // row y = y0 + r - 2 from rows y - 1 (A), y (B), y + 1 (C); e = (ex, ey)
            // comes from row y - ey, column x - ex
            const int A = (r - 2) % 3, B = (r - 1) % 3, C = r % 3;
            float g[9];
            g[0] = post[B][0][t];
            g[1] = post[B][1][t - 1];
            g[2] = post[A][2][t];
            g[3] = post[B][3][t + 1];
            g[4] = post[C][4][t];
            g[5] = post[A][5][t - 1];
            g[6] = post[A][6][t + 1];
            g[7] = post[C][7][t + 1];
            g[8] = post[C][8][t - 1];
            const size_t n = (size_t)(y0 + r - 2) * nx + xo;
#pragma unroll
            for (int i = 0; i < 9; ++i) a.fout[i * plane + n] = g[i];
            const df rr = sum9_exact(g);
            a.rh[n] = rr.hi;
            a.rl[n] = rr.lo;
        }
    }
    ring_wait_groups<0>();
    if (!ok) raise_flag(a.st, FLAG_RHO, a.st->t);
}

// Batched: block b belongs to instance map[b]; its warps continue that
// instance's warp numbering from the instance's first block.  Held to 48
// registers like the lone kernel (reading the instance's arguments took it to
// 64, eight blocks per SM instead of ten).
template <bool MRT>
__global__ void __launch_bounds__(kSwWarps * 32, 10)
    k_cs_mixed_batch(const CsBatchInst* __restrict__ d, const int* __restrict__ map, int from) {
    const CsBatchInst& D = d[map[blockIdx.x]];
    CsArgs a = D.a;
    a.fin = D.f[from];
    a.fout = D.f[1 - from];
    cs_mixed_body<MRT, false>(a, ((int)blockIdx.x - D.blk0) * kSwWarps + (threadIdx.x >> 5));
}

// f = f^eq(rho, u) in FP64, stored as FP32; rho = DF sum of the stored floats.
__global__ void k_init_mixed(const double* __restrict__ rho, const double* __restrict__ ux,
                             const double* __restrict__ uy, float* __restrict__ f,
                             float* __restrict__ rh, float* __restrict__ rl, size_t N,
                             size_t plane) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const double r = rho[n];
        const double u = ux ? ux[n] : 0.0, v = uy ? uy[n] : 0.0;
        const double uu = u * u + v * v;
        float g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double eu = ex(i) * u + ey(i) * v;
            const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
            g[i] = (float)(w * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
            f[i * plane + n] = g[i];
        }
        const df s = sum9_exact(g);
        rh[n] = s.hi;
        rl[n] = s.lo;
    }
}

__global__ void k_rho_from_f_mixed(const float* __restrict__ f, float* __restrict__ rh,
                                   float* __restrict__ rl, size_t N, size_t plane) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        float g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = f[i * plane + n];
        const df s = sum9_exact(g);
        rh[n] = s.hi;
        rl[n] = s.lo;
    }
}

// FP64 outputs of the mixed state: rho = hi + lo, v = u + F/(2 rho), mu-hat.
__global__ void k_macro_mixed(const float* __restrict__ f, const float* __restrict__ rh,
                              const float* __restrict__ rl, const float* __restrict__ Fx,
                              const float* __restrict__ Fy, double* rho_o, double* vx, double* vy,
                              size_t N, size_t plane) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        double g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = (double)f[i * plane + n];
        const double r = (double)rh[n] + (double)rl[n];
        const double jx = (g[1] + g[5] + g[8]) - (g[3] + g[6] + g[7]);
        const double jy = (g[2] + g[5] + g[6]) - (g[4] + g[7] + g[8]);
        if (rho_o) rho_o[n] = r;
        if (vx) vx[n] = (jx + 0.5 * (double)Fx[n]) / r;
        if (vy) vy[n] = (jy + 0.5 * (double)Fy[n]) / r;
    }
}

// Chemical potential of the mixed path, pointwise after the line solves of rho
// (mu_node, eos.cuh), written over d_xx rho, which nothing needs afterwards.
// Chunks of four nodes (16-byte loads and stores: the planes are 256-byte
// aligned), chunk c0, c0 + stride, ...; a short last chunk node by node.
__device__ __forceinline__ void mu_mixed_body(const float* __restrict__ rh, float* dxx_mu,
                                              const float* __restrict__ dyy, size_t N,
                                              const MuConstF& p, DevState* __restrict__ st,
                                              size_t c0, size_t stride) {
    const int64_t t = st->t;
    const bool capped = t < p.cap_steps;
    bool bad = false;
    const size_t nch = (N + 3) / 4;
    for (size_t c = c0; c < nch; c += stride) {
        const size_t n = 4 * c;
        if (n + 4 <= N) {
            const float4 r = *reinterpret_cast<const float4*>(rh + n);
            const float4 x = *reinterpret_cast<const float4*>(dxx_mu + n);
            const float4 y = *reinterpret_cast<const float4*>(dyy + n);
            float4 m;
            m.x = mu_node(r.x, x.x, y.x, p, capped, bad);
            m.y = mu_node(r.y, x.y, y.y, p, capped, bad);
            m.z = mu_node(r.z, x.z, y.z, p, capped, bad);
            m.w = mu_node(r.w, x.w, y.w, p, capped, bad);
            *reinterpret_cast<float4*>(dxx_mu + n) = m;
        } else {
            for (size_t q = n; q < N; ++q)
                dxx_mu[q] = mu_node(rh[q], dxx_mu[q], dyy[q], p, capped, bad);
        }
    }
    if (bad) raise_flag(st, FLAG_EOS, t);
}

__global__ void k_mu_mixed(const float* __restrict__ rh, float* dxx_mu,
                           const float* __restrict__ dyy, size_t N, MuConstF p,
                           DevState* __restrict__ st) {
    pdl_prologue();
    mu_mixed_body(rh, dxx_mu, dyy, N, p, st, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                  (size_t)gridDim.x * blockDim.x);
}

// Batched: blocks of kMuBatchT threads, four nodes per thread, mapped to instances.
__global__ void __launch_bounds__(kMuBatchT)
    k_mu_mixed_batch(const MuBatchInst* __restrict__ d, const int* __restrict__ map) {
    const MuBatchInst& D = d[map[blockIdx.x]];
    const size_t c = ((size_t)blockIdx.x - D.blk0) * kMuBatchT + threadIdx.x;
    mu_mixed_body(D.rh, D.mu, D.dyy, D.N, D.c, D.st, c, (D.N + 3) / 4);
}

constexpr int kDiagT = 256;

__global__ void __launch_bounds__(kDiagT)
    k_diag_mixed(const float* __restrict__ f, const float* __restrict__ rh,
                 const float* __restrict__ rl, const float* __restrict__ Fx,
                 const float* __restrict__ Fy, size_t N, size_t plane,
                 double* __restrict__ partials) {
    double s = 0.0, vmax = 0.0, rmin = DBL_MAX, rmax = -DBL_MAX;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        double g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = (double)f[i * plane + n];
        const double r = (double)rh[n] + (double)rl[n];
        const double jx = (g[1] + g[5] + g[8]) - (g[3] + g[6] + g[7]);
        const double jy = (g[2] + g[5] + g[6]) - (g[4] + g[7] + g[8]);
        const double u = (jx + 0.5 * (double)Fx[n]) / r, v = (jy + 0.5 * (double)Fy[n]) / r;
        s += r;
        vmax = fmax(vmax, sqrt(u * u + v * v));
        rmin = fmin(rmin, r);
        rmax = fmax(rmax, r);
    }
    __shared__ double sh[4][kDiagT];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = vmax;
    sh[2][threadIdx.x] = rmin;
    sh[3][threadIdx.x] = rmax;
    __syncthreads();
    for (int w = kDiagT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) partials[4 * blockIdx.x + q] = sh[q][0];
}

inline unsigned grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 65535 * 16 ? (b ? b : 1) : 65535 * 16);
}

}  // namespace

bool& launch_pdl_on() {
    thread_local bool on = true;
    return on;
}

CsArgs cs_mixed_args(const float* fin, float* fout, const float* Fx, const float* Fy,
                     float* rh, float* rl, int nx, int ny, size_t plane, double omega,
                     const MrtRates* mrt, DevState* st, int rows, const Walls& walls) {
    // rows per warp: 32 on large grids, fewer on small ones to keep >= ~4k warps
    const int nstrips = (nx + 29) / 30;
    if (rows <= 0) {
        rows = 32;
        while (rows > 8 && (long long)nstrips * ((ny + rows - 1) / rows) < 4096) rows /= 2;
    }
    CsArgs a{fin, fout, Fx, Fy, rh, rl, nx, ny, plane, (float)omega, nstrips,
             (ny + rows - 1) / rows, rows, st, mrt ? 1 : 0,
             mrt ? (float)mrt->se : 0.0f, mrt ? (float)mrt->seps : 0.0f,
             mrt ? (float)mrt->sq : 0.0f, walls.on ? 1 : 0,
             {(float)(walls.u[0] / 6.0), (float)(walls.u[1] / 6.0)}};
    return a;
}

// Below this many nodes the sliding window is faster (1024^2: 20.5 us against
// 22.5; 2048^2: 65.5 against 67.5; its 40 warps an SM hide latency better than
// the ring's 20 when the grid is a wave or two of blocks); at and above it the
// ring is (4096^2: 240 us against 263).
constexpr long long kRingMinNodes = 1ll << 23;

bool cs_ring_fits(const CsArgs& a) {
    auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    return !a.walls && a.nx % 4 == 0 && a.nx >= kRingT && a.plane % 4 == 0 && al16(a.fin) &&
           al16(a.Fx) && al16(a.Fy);
}

// Row-ring arguments: strips of kRingW columns; `rows` rows a block (0: 8, the
// fastest of 8, 16 and 32 at 1024^2 and 4096^2)
CsArgs cs_ring_args(CsArgs a, int rows) {
    a.nstrips = (a.nx + kRingW - 1) / kRingW;
    if (rows <= 0) rows = 8;
    a.rows = rows;
    a.nseg = (a.ny + rows - 1) / rows;
    return a;
}

int cs_mixed_blocks(const CsArgs& a) {
    const long long warps = (long long)a.nstrips * a.nseg;
    return (int)((warps + kSwWarps - 1) / kSwWarps);
}

cudaError_t launch_cs_mixed_args(const CsArgs& a, cudaStream_t s) {
    const int nb = cs_mixed_blocks(a);
    if (a.mrt && a.walls) return launch_pdl(k_cs_mixed_sw_walls<true>, nb, kSwWarps * 32, 0, s, a);
    if (a.mrt) return launch_pdl(k_cs_mixed_sw<true>, nb, kSwWarps * 32, 0, s, a);
    if (a.walls) return launch_pdl(k_cs_mixed_sw_walls<false>, nb, kSwWarps * 32, 0, s, a);
    return launch_pdl(k_cs_mixed_sw<false>, nb, kSwWarps * 32, 0, s, a);
}

cudaError_t launch_cs_mixed(const float* fin, float* fout, const float* Fx, const float* Fy,
                            float* rh, float* rl, int nx, int ny, size_t plane, double omega,
                            const MrtRates* mrt, DevState* st, cudaStream_t s,
                            const Walls& walls, int ring_rows) {
    const CsArgs a =
        cs_mixed_args(fin, fout, Fx, Fy, rh, rl, nx, ny, plane, omega, mrt, st, 0, walls);
    if (!cs_ring_used(nx, ny, plane, fin, Fx, Fy, walls.on, ring_rows))
        return launch_cs_mixed_args(a, s);
    const CsArgs r = cs_ring_args(a, ring_rows);
    const unsigned nb = (unsigned)(r.nstrips * r.nseg);
    return r.mrt ? launch_pdl(k_cs_mixed_ring<true>, nb, kRingT, 0, s, r)
                 : launch_pdl(k_cs_mixed_ring<false>, nb, kRingT, 0, s, r);
}

bool cs_ring_used(int nx, int ny, size_t plane, const void* fin, const void* Fx,
                  const void* Fy, bool walls, int ring_rows) {
    if (ring_rows < 0 || (ring_rows == 0 && (long long)nx * ny < kRingMinNodes)) return false;
    CsArgs a{};
    a.fin = (const float*)fin;
    a.Fx = (const float*)Fx;
    a.Fy = (const float*)Fy;
    a.nx = nx;
    a.ny = ny;
    a.plane = plane;
    a.walls = walls ? 1 : 0;
    return cs_ring_fits(a);
}

cudaError_t launch_cs_mixed_batch(const CsBatchInst* d, const int* map, int nblocks, int from,
                                  bool mrt, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    if (mrt)
        k_cs_mixed_batch<true><<<nblocks, kSwWarps * 32, 0, s>>>(d, map, from);
    else
        k_cs_mixed_batch<false><<<nblocks, kSwWarps * 32, 0, s>>>(d, map, from);
    return cudaGetLastError();
}

cudaError_t launch_init_mixed(const double* rho, const double* ux, const double* uy, float* f,
                              float* rh, float* rl, int nx, int ny, size_t plane,
                              cudaStream_t s) {
    const size_t N = (size_t)nx * ny;
    k_init_mixed<<<grid_for(N, 256), 256, 0, s>>>(rho, ux, uy, f, rh, rl, N, plane);
    return cudaGetLastError();
}

cudaError_t launch_rho_from_f_mixed(const float* f, float* rh, float* rl, int nx, int ny,
                                    size_t plane, cudaStream_t s) {
    const size_t N = (size_t)nx * ny;
    k_rho_from_f_mixed<<<grid_for(N, 256), 256, 0, s>>>(f, rh, rl, N, plane);
    return cudaGetLastError();
}

cudaError_t launch_macro_mixed(const float* f, const float* rh, const float* rl,
                               const float* Fx, const float* Fy, double* rho, double* vx,
                               double* vy, int nx, int ny, size_t plane, cudaStream_t s) {
    const size_t N = (size_t)nx * ny;
    k_macro_mixed<<<grid_for(N, 256), 256, 0, s>>>(f, rh, rl, Fx, Fy, rho, vx, vy, N, plane);
    return cudaGetLastError();
}

MuConstF mu_mixed_const(const PhysParams& p) {
    return MuConstF{eos_const<float>(p), (float)p.k2, (float)p.kappa,
                    (float)fmin(p.mu_cap, (double)FLT_MAX), p.cap_steps};
}

cudaError_t launch_mu_mixed(const float* rh, float* dxx_mu, const float* dyy, int nx, int ny,
                            const PhysParams& p, DevState* st, cudaStream_t s) {
    const size_t N = (size_t)nx * ny;
    return launch_pdl(k_mu_mixed, grid_for((N + 3) / 4, 256), 256, 0, s, rh, dxx_mu, dyy, N,
                      mu_mixed_const(p), st);
}

cudaError_t launch_mu_mixed_batch(const MuBatchInst* d, const int* map, int nblocks,
                                  cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    k_mu_mixed_batch<<<nblocks, kMuBatchT, 0, s>>>(d, map);
    return cudaGetLastError();
}

cudaError_t launch_diag_mixed(const float* f, const float* rh, const float* rl, const float* Fx,
                              const float* Fy, int nx, int ny, size_t plane, double* partials,
                              int nparts, DevState* st, cudaStream_t s) {
    const size_t N = (size_t)nx * ny;
    k_diag_mixed<<<nparts, kDiagT, 0, s>>>(f, rh, rl, Fx, Fy, N, plane, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_diag_final(partials, nparts, st, s);
}

}  // namespace cplbm
