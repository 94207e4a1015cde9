// cplbm_internal.cuh -- shared declarations of the CUDA library (device
// kernels, launchers and the context).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/cplbm.h"

#include <utility>

namespace cplbm {

// ---- programmatic dependent launch (the single-instance mixed step) --------
// The kernels of a mixed step are each about one wave at small grids, so the gap
// between one kernel's last blocks and the next kernel's first is a visible part
// of the step.  Launched with the programmatic-serialization attribute, a kernel
// lets the next one be scheduled once all of its own blocks have started
// (launch_dependents), and waits, before touching memory, until the previous
// kernel has completed and its writes are visible (wait).  The next kernel's
// blocks thus become resident during this one's tail instead of after it.  Both
// instructions are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// Whether launch_pdl sets the attribute: chosen per context by whoever enqueues
// (the host thread that enqueues a step sets it first; enqueueing is synchronous).
bool& launch_pdl_on();

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = launch_pdl_on() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

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
    FLAG_EOS = 2u,   // EOS pass: rho <= 0, the EOS pole with the upper limit off,
                     // or mu not finite
    FLAG_STAGE = 4u, // a line window's tensor copy did not arrive within the
                     // bounded wait (the block gave up; the step is void)
};

// Physical parameters the kernels need.
struct PhysParams {
    int eos;             // LBM_EOS_* (Sec. 3.2)
    double alpha;        // alpha(T) of Eqs. 16-19 at this T (1 for CS and VDW)
    double T, a, b, R;   // EOS constants, T absolute
    double k2;           // k^2 (Eq. 33)
    double kappa;        // kappa-hat (Eq. 33)
    double omega;        // 1 / tau (Eq. 1)
    double mu_cap;       // k^2 * mu_max (mesh-space limit, Sec. 5.6)
    int64_t cap_steps;   // limit active while t < cap_steps
};

// MRT relaxation rates of Eq. 4 other than s_v = 1/tau (NULL pointer: BGK).
struct MrtRates {
    double se, seps, sq;
};

// Solid walls below row 0 and above row ny-1 (Sec. 5.5), halfway bounce-back;
// u: the x-velocities of the bottom and the top wall (a moving frame).
struct Walls {
    bool on = false;
    double u[2] = {0.0, 0.0};
};

// Launchers (all asynchronous on `s`).  Fields are FP64 [ny][nx]; populations
// are [9][plane] of TF with plane >= nx*ny.
template <typename TF>
cudaError_t launch_collide_stream(const TF* fin, TF* fout, const double* Fx, const double* Fy,
                                  double* rho_out, int nx, int ny, size_t plane, double omega,
                                  const MrtRates* mrt, DevState* st, cudaStream_t s,
                                  const Walls& walls = Walls());

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

cudaError_t launch_diag_final(const double* partials, int nparts, DevState* st, cudaStream_t s);

// ---- mixed precision path (kernels_mixed.cu) ------------------------------
// ring_rows: -1 = the sliding-window kernel; 0 = the row-ring kernel where the
// grid allows it (periodic, nx a multiple of 4 and >= 128, aligned planes), with
// its default rows a block; > 0 = the row-ring kernel with that many rows a block
cudaError_t launch_cs_mixed(const float* fin, float* fout, const float* Fx, const float* Fy,
                            float* rh, float* rl, int nx, int ny, size_t plane, double omega,
                            const MrtRates* mrt, DevState* st, cudaStream_t s,
                            const Walls& walls = Walls(), int ring_rows = -1);
// whether launch_cs_mixed with these arguments runs the row-ring kernel
bool cs_ring_used(int nx, int ny, size_t plane, const void* fin, const void* Fx,
                  const void* Fy, bool walls, int ring_rows);
cudaError_t launch_init_mixed(const double* rho, const double* ux, const double* uy, float* f,
                              float* rh, float* rl, int nx, int ny, size_t plane,
                              cudaStream_t s);
cudaError_t launch_rho_from_f_mixed(const float* f, float* rh, float* rl, int nx, int ny,
                                    size_t plane, cudaStream_t s);
cudaError_t launch_macro_mixed(const float* f, const float* rh, const float* rl,
                               const float* Fx, const float* Fy, double* rho, double* vx,
                               double* vy, int nx, int ny, size_t plane, cudaStream_t s);
cudaError_t launch_diag_mixed(const float* f, const float* rh, const float* rl, const float* Fx,
                              const float* Fy, int nx, int ny, size_t plane, double* partials,
                              int nparts, DevState* st, cudaStream_t s);

// ---- batched mixed path: per-instance argument blocks -----------------------
// A batch runs many independent instances (each its own grid, temperature,
// tau, k, kappa and state block) through the same four passes, one launch per
// pass for the whole batch.  Every launch reads, per block, the instance index
// from a block map and that instance's argument block; inside an instance the
// work is the single-instance kernel's, block for block.

// Collide-stream arguments of one instance (mixed path).
struct CsArgs {
    const float* fin;
    float* fout;
    const float* Fx;
    const float* Fy;
    float* rh;
    float* rl;
    int nx, ny;
    size_t plane;
    float omega;
    int nstrips, nseg, rows;  // warp strips of 30 columns x `rows` rows
    DevState* st;
    int mrt;                  // 0: BGK (Eq. 1); 1: MRT (Eq. 4) with the rates below
    float se, seps, sq;
    int walls;                // 1: halfway bounce-back below row 0 and above row ny-1
    float uw6[2];             // bottom / top wall x-velocity over 6 (moving walls)
};
struct CsBatchInst {
    CsArgs a;      // fin / fout are taken from f[] by the launch's `from`
    float* f[2];
    int blk0;      // first block of this instance in the launch
};
// FP32 constants of the chemical potential, converted on the host: FP64 -> FP32
// conversions run on the FP64 pipe, which a per-thread conversion would make the
// bottleneck of the pointwise kernel.
template <class T>
struct EosC {
    int kind;   // LBM_EOS_*
    T rt;       // R T
    T a2;       // 2 a (CS, VDW)
    T b;        // b (cubic EOSs) or b / 4 (CS)
    T aal;      // a alpha(T) (RK, RKS, PR)
    T clog;     // a alpha / b (RK, RKS) or a alpha / (2 sqrt 2 b) (PR)
};
struct MuConstF {
    EosC<float> e;
    float k2, kappa, cap;
    long long cap_steps;
};
// The EOS constants of PhysParams in arithmetic T (host).
template <class T>
EosC<T> eos_const(const PhysParams& p) {
    EosC<T> c;
    c.kind = p.eos;
    c.rt = (T)(p.R * p.T);
    c.a2 = (T)(2 * p.a);
    c.b = (T)(p.eos == LBM_EOS_CS ? 0.25 * p.b : p.b);
    c.aal = (T)(p.a * p.alpha);
    c.clog = (T)(p.eos == LBM_EOS_PR ? p.a * p.alpha / (2 * 1.4142135623730951 * p.b)
                                     : p.a * p.alpha / p.b);
    return c;
}
constexpr int kMuBatchT = 256;  // threads per block of the batched mu-hat pass (4 nodes each)
struct MuBatchInst {
    const float* rh;
    float* mu;  // holds d_xx rho on entry
    const float* dyy;
    size_t N;
    MuConstF c;
    DevState* st;
    int blk0;
};
// Pointers and sizes of one instance's mixed fields, for the batched line passes.
struct MixedLinesView {
    const float* rh;
    const float* rl;
    float *dxr, *dyr, *dxx, *dyy;  // dxx holds mu-hat after the mu pass
    float *Fx, *Fy;
    int nx, ny;
    DevState* st;
};

CsArgs cs_mixed_args(const float* fin, float* fout, const float* Fx, const float* Fy,
                     float* rh, float* rl, int nx, int ny, size_t plane, double omega,
                     const MrtRates* mrt, DevState* st,
                     int rows,  // rows <= 0: the default choice
                     const Walls& walls = Walls());
int cs_mixed_blocks(const CsArgs& a);
cudaError_t launch_cs_mixed_args(const CsArgs& a, cudaStream_t s);
cudaError_t launch_cs_mixed_batch(const CsBatchInst* d, const int* map, int nblocks, int from,
                                  bool mrt, cudaStream_t s);
MuConstF mu_mixed_const(const PhysParams& p);
cudaError_t launch_mu_mixed_batch(const MuBatchInst* d, const int* map, int nblocks,
                                  cudaStream_t s);
// Line passes: descriptor size per instance, blocks per instance, descriptor
// written to host memory (copied to the device by the caller), the launches.
enum class LineBatchKind {
    kRhoDF,   // x|y lines of the density, double-float where a window needs it
    kRhoF32,  // x|y lines of the density in FP32 (the hi part only)
    kForce,   // x|y lines of mu-hat with the force epilogue
};
size_t lines_batch_desc_bytes(LineBatchKind kind);
// nl: lines per block, 8 or 16 (the FP32 kinds; the double-float density lines
// always take 8).  Results do not depend on it.
int lines_batch_blocks(int nx, int ny, int order, LineBatchKind kind, int nl = 8);
void lines_batch_fill(LineBatchKind kind, const MixedLinesView& v, int order, int blk0,
                      void* host_dst, int nl = 8);
cudaError_t lines_batch_launch(LineBatchKind kind, const void* d_desc, const int* map,
                               int nblocks, int order, int bump, cudaStream_t s, int nl = 8);

// Below this Maxwell density ratio the mixed path solves the density's lines in
// FP32 (measured: coexistence densities within 2e-4 of the FP64 path); at and
// above it, in double-float wherever a window spans more than a factor 32.
constexpr double kDfRatio = 1e4;

// Warp-cooperative compact-FD line solves (kernels_lines.cu).  With walls_y the
// y-lines are extended evenly about both walls (a periodic line of period
// 2 ny, the first ghost equal to its fluid neighbour, Sec. 5.5).  axis 0: lines
// along x, 1: along y.  Passes 2-5 of the FP64 path and of the mixed path, and
// the stand-alone derivatives.
cudaError_t lines_fp64_rho_x(const double* rho, double* dxr, double* dxx, int nx, int ny,
                             int order, DevState* st, int bump, cudaStream_t s);
cudaError_t lines_fp64_rho_y_mu(const double* rho, const double* dxx, double* dyr, double* mu,
                                int nx, int ny, int order, const PhysParams& p, DevState* st,
                                cudaStream_t s, bool walls_y = false);
cudaError_t lines_fp64_force(const double* mu, const double* rho, const double* dr, double* F,
                             int nx, int ny, int axis, int order, cudaStream_t s,
                             bool walls_y = false);
cudaError_t lines_fp64_plain(const double* u, double* d1, double* d2, int nx, int ny, int axis,
                             int order, cudaStream_t s);
// Mixed path, merged launches: the x- and y-lines of rho together (first and
// second derivatives); then, after launch_mu_mixed, the x- and y-lines of
// mu-hat together with the force epilogue.
cudaError_t lines_mixed_rho_xy(const float* rh, const float* rl, float* dxr, float* dxx,
                               float* dyr, float* dyy, int nx, int ny, int order, DevState* st,
                               int bump, cudaStream_t s, bool walls_y = false);
// The same in FP32 on the hi part of the density (below kDfRatio).
cudaError_t lines_mixed_rho_xy_f32(const float* rh, float* dxr, float* dxx, float* dyr,
                                   float* dyy, int nx, int ny, int order, DevState* st, int bump,
                                   cudaStream_t s, bool walls_y = false);
cudaError_t lines_mixed_force_xy(const float* mu, const float* rh, const float* dxr,
                                 const float* dyr, float* Fx, float* Fy, int nx, int ny,
                                 int order, cudaStream_t s, bool walls_y = false,
                                 DevState* st = nullptr);
// mu-hat = k^2 mu0(rho) - kappa (d_xx + d_yy) rho (Eqs. 21, 33, Sec. 5.6), FP32,
// written over d_xx rho (`dxx_mu`); flags bad values.
cudaError_t launch_mu_mixed(const float* rh, float* dxx_mu, const float* dyy, int nx, int ny,
                            const PhysParams& p, DevState* st, cudaStream_t s);
cudaError_t lines_mixed_plain(const float* uh, const float* ul, float* d1, float* d2, int nx,
                              int ny, int axis, int order, cudaStream_t s);

// Host thermodynamics of the product library (independent of the oracle), for
// the EOS kinds LBM_EOS_* (Sec. 3.2).  Return 0 or -1 (invalid arguments, or
// T outside (0, T_c) for the Maxwell pair).
int eos_critical(int kind, double a, double b, double R, double* Tc, double* rhoc);
double eos_alpha(int kind, double a, double b, double R, double omega, double T);
int eos_maxwell(int kind, double a, double b, double R, double omega, double T,
                double* rho_g, double* rho_l);

}  // namespace cplbm
