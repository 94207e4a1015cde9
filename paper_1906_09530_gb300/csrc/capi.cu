// capi.cu -- the C ABI of include/cplbm.h: argument checks, workspace layout,
// the per-step pass schedule (captured in CUDA graphs), host<->device copies,
// error flag and bounded waits.
//
// FP64 path: one time step is five device passes (all on the caller's stream):
//   1 collide-stream      f^t, F^t           -> f^{t+1}, rho^{t+1}      Eqs. 1-5
//   2 x-lines of rho      rho                -> d_x rho, d_xx rho       Eqs. 37-39
//   3 y-lines of rho      rho, d_xx rho      -> d_y rho, mu-hat         Eqs. 21, 33, Sec. 5.6
//   4 x-lines of mu-hat   mu, rho, d_x rho   -> F_x                     Eq. 12
//   5 y-lines of mu-hat   mu, rho, d_y rho   -> F_y                     Eq. 12
// Mixed path: four passes -- collide-stream; the x- and y-lines of rho in one
// launch (d_x, d_xx, d_y, d_yy rho); mu-hat pointwise (stored over d_xx rho);
// the x- and y-lines of mu-hat in one launch with the force epilogue.
// Passes after the first compute the force of the new time level;
// lbm_set_fields runs them once on the initial density.  Each needs its input
// complete over whole lines or all nodes, so they are separate launches.
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>

#include "cplbm_internal.cuh"

using namespace cplbm;

struct lbm_ctx {
    int dev;
    int nx, ny;
    size_t N, plane;
    int prec, fd_order;
    bool rho_df;  // mixed: density lines in double-float (else FP32)
    bool walls_y; // solid walls below row 0 and above row ny-1 (Sec. 5.5)
    Walls walls;  // the same, with the walls' x-velocities, for the collide pass
    bool mrt;     // MRT collision (Eq. 4) with the rates below
    int ring_rows; // mixed collide-stream form: -1 sliding window, 0 by grid size,
                   // > 0 row ring with that many rows a block
    // programmatic dependent launch between the mixed step's kernels, chosen
    // separately for direct launches and for the launches captured in graphs;
    // pdl_now is what the passes being enqueued use
    bool pdl_direct, pdl_graph, pdl_now;
    bool single_graph;  // a lone step (lbm_step_async of 1, an odd last step) from a graph
    MrtRates rates;
    double T, Tc, rhoc, kappa, tau, k;
    double mu_max;
    int64_t mu_cap_steps;
    PhysParams phys;
    cudaStream_t stream;      // caller's stream
    cudaStream_t cap_stream;  // private, for graph capture only
    cudaEvent_t ev;
    cudaEvent_t tev[6];  // timing events of lbm_step_timed
    char* ws;
    size_t ws_bytes;
    void* f[2];
    int cur;
    double *rho, *dxr, *dyr, *dxx, *mu, *Fx, *Fy;  // FP64 path
    // mixed path: density as hi/lo floats, the rest FP32
    float *m_rh, *m_rl, *m_dxr, *m_dyr, *m_dxx, *m_dyy, *m_Fx, *m_Fy;
    double* partials;
    int nparts;
    DevState* dst;   // device
    DevState* hst;   // pinned host mirror
    int64_t t;
    int64_t failed;
    bool ready;      // fields set
    cudaGraphExec_t graph[2];    // two steps, starting from f[0] / f[1]
    cudaGraphExec_t graph16[2];  // kLongGraph steps, likewise (fewer graph launches)
    cudaGraphExec_t graph1[2];   // one step, for single steps when single_graph is set
    double timeout_s;
};

namespace {

constexpr size_t kAlign = 256;
constexpr int kParts = 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    size_t plane, f_bytes, field_bytes;
    size_t off_f0, off_f1, off_fields, off_parts, off_state, total;
};

bool grid_ok(const lbm_grid* g) { return g && g->nx >= 8 && g->ny >= 8; }
bool rate_ok(double s) { return s > 0 && s < 2; }
bool opts_ok(const lbm_opts* o) {
    return o &&
           (o->prec == LBM_PREC_FP64 || o->prec == LBM_PREC_MIXED ||
            o->prec == LBM_PREC_MIXED_DF) &&
           (o->collision == LBM_COLLIDE_BGK ||
            (o->collision == LBM_COLLIDE_MRT && rate_ok(o->s_e) && rate_ok(o->s_eps) &&
             rate_ok(o->s_q))) &&
           (o->fd_order == 4 || o->fd_order == 6) && !std::isnan(o->mu_max);
}

// Workspace: two population buffers, then the fields (FP64 path: seven FP64
// planes; mixed path: eight FP32 planes), reduction partials, device state.
Layout layout(int nx, int ny, int prec) {
    Layout L;
    const size_t N = (size_t)nx * ny;
    L.plane = align_up(N, 64);
    const bool f64 = prec == LBM_PREC_FP64;
    const size_t tf = f64 ? sizeof(double) : sizeof(float);
    L.f_bytes = align_up(9 * L.plane * tf, kAlign);
    L.field_bytes = align_up(L.plane * tf, kAlign);
    L.off_f0 = 0;
    L.off_f1 = L.off_f0 + L.f_bytes;
    L.off_fields = L.off_f1 + L.f_bytes;
    L.off_parts = L.off_fields + (f64 ? 7 : 8) * L.field_bytes;
    L.off_state = L.off_parts + align_up(4 * kParts * sizeof(double), kAlign);
    L.total = L.off_state + align_up(sizeof(DevState), kAlign);
    return L;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return LBM_ECUDA;  \
    } while (0)

bool is_fp64(const lbm_ctx* c) { return c->prec == LBM_PREC_FP64; }

lbm_status use_dev(lbm_ctx* c) {
    CK(cudaSetDevice(c->dev));
    return LBM_OK;
}

// Passes 2-5 on the current density.  `timed` records an event after each.
lbm_status enqueue_force(lbm_ctx* c, cudaStream_t s, int bump, cudaEvent_t* ev = nullptr) {
    const int nx = c->nx, ny = c->ny, o = c->fd_order;
    launch_pdl_on() = c->pdl_now;
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    if (!is_fp64(c)) {
        // x|y lines of rho together, mu-hat pointwise, x|y lines of mu-hat + force
        if (c->rho_df)
            CK(lines_mixed_rho_xy(c->m_rh, c->m_rl, c->m_dxr, c->m_dxx, c->m_dyr, c->m_dyy, nx,
                                  ny, o, c->dst, bump, s, c->walls_y));
        else
            CK(lines_mixed_rho_xy_f32(c->m_rh, c->m_dxr, c->m_dxx, c->m_dyr, c->m_dyy, nx, ny, o,
                                      c->dst, bump, s, c->walls_y));
        CK(mark(0));
        CK(launch_mu_mixed(c->m_rh, c->m_dxx, c->m_dyy, nx, ny, c->phys, c->dst, s));
        CK(mark(1));
        CK(lines_mixed_force_xy(c->m_dxx, c->m_rh, c->m_dxr, c->m_dyr, c->m_Fx, c->m_Fy, nx, ny,
                                o, s, c->walls_y, c->dst));
        CK(mark(2));
        CK(mark(3));
        return LBM_OK;
    }
    CK(lines_fp64_rho_x(c->rho, c->dxr, c->dxx, nx, ny, o, c->dst, bump, s));
    CK(mark(0));
    CK(lines_fp64_rho_y_mu(c->rho, c->dxx, c->dyr, c->mu, nx, ny, o, c->phys, c->dst, s,
                           c->walls_y));
    CK(mark(1));
    CK(lines_fp64_force(c->mu, c->rho, c->dxr, c->Fx, nx, ny, 0, o, s));
    CK(mark(2));
    CK(lines_fp64_force(c->mu, c->rho, c->dyr, c->Fy, nx, ny, 1, o, s, c->walls_y));
    CK(mark(3));
    return LBM_OK;
}

// Pass 1 from f[from] into f[1-from].
lbm_status enqueue_collide(lbm_ctx* c, cudaStream_t s, int from) {
    const int to = 1 - from;
    launch_pdl_on() = c->pdl_now;
    if (is_fp64(c))
        CK(launch_collide_stream<double>((const double*)c->f[from], (double*)c->f[to], c->Fx,
                                         c->Fy, c->rho, c->nx, c->ny, c->plane,
                                         c->phys.omega, c->mrt ? &c->rates : nullptr, c->dst,
                                         s, c->walls));
    else
        CK(launch_cs_mixed((const float*)c->f[from], (float*)c->f[to], c->m_Fx, c->m_Fy,
                           c->m_rh, c->m_rl, c->nx, c->ny, c->plane, c->phys.omega,
                           c->mrt ? &c->rates : nullptr, c->dst, s, c->walls, c->ring_rows));
    return LBM_OK;
}

// One full time step starting from f[from]; leaves the state in f[1-from].
lbm_status enqueue_step(lbm_ctx* c, cudaStream_t s, int from) {
    lbm_status st = enqueue_collide(c, s, from);
    if (st) return st;
    return enqueue_force(c, s, 1);
}

// Steps in the long graph: even, so a replay ends on the buffer it started from.
constexpr int kLongGraph = 16;

void drop_graphs(lbm_ctx* c) {
    for (int i = 0; i < 2; ++i)
        for (cudaGraphExec_t* gp : {&c->graph[i], &c->graph16[i], &c->graph1[i]})
            if (*gp) {
                cudaGraphExecDestroy(*gp);
                *gp = nullptr;
            }
}

// Capture `steps` (even) time steps starting from f[from] into *out.
lbm_status build_graph(lbm_ctx* c, int from, int steps, cudaGraphExec_t* out) {
    if (*out) return LBM_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    lbm_status st = LBM_OK;
    c->pdl_now = c->pdl_graph;
    for (int i = 0; i < steps && st == LBM_OK; ++i)
        st = enqueue_step(c, c->cap_stream, (from + i) & 1);
    c->pdl_now = c->pdl_direct;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return LBM_ECUDA;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

// Wait for everything enqueued on the stream, with the context's time limit.
lbm_status wait_stream(lbm_ctx* c) {
    CK(cudaEventRecord(c->ev, c->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaEventQuery(c->ev);
        if (q == cudaSuccess) return LBM_OK;
        if (q != cudaErrorNotReady) return LBM_ECUDA;
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > c->timeout_s) return LBM_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
    }
}

// Read back the device state block and translate the error flag.
lbm_status read_state(lbm_ctx* c) {
    CK(cudaMemcpyAsync(c->hst, c->dst, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    lbm_status w = wait_stream(c);
    if (w != LBM_OK) return w;
    if (c->hst->flag) {
        c->failed = c->hst->failed_t == ULLONG_MAX ? c->t : (int64_t)c->hst->failed_t;
        c->ready = false;
        return (c->hst->flag & FLAG_STAGE) ? LBM_ETIMEOUT : LBM_EUNSTABLE;
    }
    return LBM_OK;
}

lbm_status reset_state(lbm_ctx* c, int64_t t) {
    DevState h;
    std::memset(&h, 0, sizeof(h));
    h.t = t;
    h.failed_t = ULLONG_MAX;
    // the pinned mirror is the copy source; it is not touched again before the
    // stream is drained by the caller of reset_state
    *c->hst = h;
    CK(cudaMemcpyAsync(c->dst, c->hst, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    c->t = t;
    c->failed = -1;
    return LBM_OK;
}

double* staging(lbm_ctx* c) { return (double*)c->f[1 - c->cur]; }

}  // namespace

extern "C" {

const char* lbm_strerror(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "workspace too small or out of host memory";
        case LBM_ECUDA: return "CUDA runtime error";
        case LBM_EUNSTABLE: return "unstable: rho <= 0, non-finite value or EOS pole";
        case LBM_ETIMEOUT: return "device work did not finish within the time limit";
        case LBM_ENOTIMPL: return "not implemented";
    }
    return "unknown status";
}

size_t lbm_workspace_bytes(const lbm_grid* grid, const lbm_opts* opts) {
    if (!grid_ok(grid) || !opts_ok(opts)) return 0;
    return layout(grid->nx, grid->ny, opts->prec).total;
}

static bool eos_valid(const lbm_eos* eos) {
    return eos && eos->kind >= LBM_EOS_CS && eos->kind <= LBM_EOS_PR && eos->a > 0 &&
           eos->b > 0 && eos->R > 0 && std::isfinite(eos->omega);
}

lbm_status lbm_critical(const lbm_eos* eos, double* Tc, double* rhoc) {
    if (!eos_valid(eos) || !Tc || !rhoc) return LBM_EINVAL;
    return eos_critical(eos->kind, eos->a, eos->b, eos->R, Tc, rhoc) ? LBM_EINVAL : LBM_OK;
}

lbm_status lbm_maxwell(const lbm_eos* eos, double T_r, double* rho_g, double* rho_l) {
    if (!eos_valid(eos) || !rho_g || !rho_l) return LBM_EINVAL;
    if (!(T_r > 0 && T_r < 1)) return LBM_EINVAL;
    double Tc, rc;
    if (eos_critical(eos->kind, eos->a, eos->b, eos->R, &Tc, &rc)) return LBM_EINVAL;
    return eos_maxwell(eos->kind, eos->a, eos->b, eos->R, eos->omega, T_r * Tc, rho_g, rho_l)
               ? LBM_EINVAL
               : LBM_OK;
}

lbm_status lbm_init(lbm_ctx** out, const lbm_grid* grid, const lbm_eos* eos, double T_r,
                    double kappa, double tau, double mesh_coeff, const lbm_opts* opts,
                    void* d_workspace, size_t ws_bytes, void* cuda_stream) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!grid_ok(grid) || !opts_ok(opts) || !eos) return LBM_EINVAL;
    if (!grid->periodic_x) return LBM_ENOTIMPL;  // walls are built in y only
    if (!eos_valid(eos)) return LBM_EINVAL;
    if (!(T_r > 0 && T_r < 1) || !(kappa > 0) || !(tau > 0.5) ||
        !(mesh_coeff > 0 && mesh_coeff <= 1))
        return LBM_EINVAL;
    if (!d_workspace || ((uintptr_t)d_workspace % kAlign)) return LBM_EINVAL;
    const Layout L = layout(grid->nx, grid->ny, opts->prec);
    if (ws_bytes < L.total) return LBM_ENOMEM;
    double Tc, rc;
    if (eos_critical(eos->kind, eos->a, eos->b, eos->R, &Tc, &rc)) return LBM_EINVAL;

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    std::memset((void*)c, 0, sizeof(*c));
    if (cudaGetDevice(&c->dev) != cudaSuccess) {
        delete c;
        return LBM_ECUDA;
    }
    c->nx = grid->nx;
    c->ny = grid->ny;
    c->N = (size_t)grid->nx * grid->ny;
    c->plane = L.plane;
    c->prec = opts->prec;
    c->fd_order = opts->fd_order;
    c->rho_df = opts->prec == LBM_PREC_MIXED_DF;
    c->mrt = opts->collision == LBM_COLLIDE_MRT;
    c->ring_rows = 0;
    c->pdl_direct = true;
    c->pdl_graph = false;
    c->pdl_now = c->pdl_direct;
    c->single_graph = true;
    c->walls_y = !grid->periodic_y;
    c->walls.on = c->walls_y;
    c->rates = MrtRates{opts->s_e, opts->s_eps, opts->s_q};
    if (opts->prec == LBM_PREC_MIXED) {
        double rg, rl;
        c->rho_df = eos_maxwell(eos->kind, eos->a, eos->b, eos->R, eos->omega, T_r * Tc, &rg,
                                &rl) != 0 ||
                    !(rl < kDfRatio * rg);
    }
    c->Tc = Tc;
    c->rhoc = rc;
    c->T = T_r * Tc;
    c->kappa = kappa;
    c->tau = tau;
    c->k = mesh_coeff;
    c->mu_max = opts->mu_max;
    c->mu_cap_steps = opts->mu_cap_steps;
    c->phys.eos = eos->kind;
    c->phys.alpha = eos_alpha(eos->kind, eos->a, eos->b, eos->R, eos->omega, c->T);
    c->phys.T = c->T;
    c->phys.a = eos->a;
    c->phys.b = eos->b;
    c->phys.R = eos->R;
    c->phys.k2 = mesh_coeff * mesh_coeff;
    c->phys.kappa = kappa;
    c->phys.omega = 1.0 / tau;
    c->phys.mu_cap = std::isinf(opts->mu_max) ? HUGE_VAL : c->phys.k2 * opts->mu_max;
    c->phys.cap_steps = opts->mu_cap_steps;
    c->stream = (cudaStream_t)cuda_stream;
    c->ws = (char*)d_workspace;
    c->ws_bytes = ws_bytes;
    c->f[0] = c->ws + L.off_f0;
    c->f[1] = c->ws + L.off_f1;
    double* fields = (double*)(c->ws + L.off_fields);
    const size_t fs = L.field_bytes / sizeof(double);
    if (opts->prec == LBM_PREC_FP64) {
        c->rho = fields;
        c->dxr = fields + fs;
        c->dyr = fields + 2 * fs;
        c->dxx = fields + 3 * fs;
        c->mu = fields + 4 * fs;
        c->Fx = fields + 5 * fs;
        c->Fy = fields + 6 * fs;
    } else {
        float* ff = (float*)fields;
        const size_t ffs = L.field_bytes / sizeof(float);
        float** slots[8] = {&c->m_rh, &c->m_rl, &c->m_dxr, &c->m_dyr,
                            &c->m_dxx, &c->m_dyy, &c->m_Fx, &c->m_Fy};
        for (int i = 0; i < 8; ++i) *slots[i] = ff + i * ffs;
    }
    c->partials = (double*)(c->ws + L.off_parts);
    c->nparts = kParts;
    c->dst = (DevState*)(c->ws + L.off_state);
    c->t = 0;
    c->failed = -1;
    c->timeout_s = 600.0;
    c->cur = 0;
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&c->hst, sizeof(DevState)) != cudaSuccess) {
        lbm_free(c);
        return LBM_ECUDA;
    }
    for (int i = 0; i < 6; ++i)
        if (cudaEventCreate(&c->tev[i]) != cudaSuccess) {
            lbm_free(c);
            return LBM_ECUDA;
        }
    *out = c;
    return LBM_OK;
}

void lbm_free(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    drop_graphs(c);
    if (c->ev) cudaEventDestroy(c->ev);
    for (int i = 0; i < 6; ++i)
        if (c->tev[i]) cudaEventDestroy(c->tev[i]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->hst) cudaFreeHost(c->hst);
    delete c;
}

lbm_status lbm_set_timeout(lbm_ctx* c, double seconds) {
    if (!c || !(seconds > 0)) return LBM_EINVAL;
    c->timeout_s = seconds;
    return LBM_OK;
}

lbm_status lbm_set_wall_velocity(lbm_ctx* c, double u_bottom, double u_top) {
    if (!c || !c->walls_y || !(std::fabs(u_bottom) < 0.5) || !(std::fabs(u_top) < 0.5))
        return LBM_EINVAL;
    c->walls.u[0] = u_bottom;
    c->walls.u[1] = u_top;
    drop_graphs(c);  // the captured collide launches hold the old velocities
    return LBM_OK;
}

int32_t lbm_path_flags(const lbm_ctx* c) {
    if (!c) return -1;
    if (c->prec == LBM_PREC_FP64) return 0;
    int32_t f = c->rho_df ? LBM_PATH_RHO_DF : 0;
    if (cs_ring_used(c->nx, c->ny, c->plane, c->f[0], c->m_Fx, c->m_Fy, c->walls_y,
                     c->ring_rows) &&
        cs_ring_used(c->nx, c->ny, c->plane, c->f[1], c->m_Fx, c->m_Fy, c->walls_y,
                     c->ring_rows))
        f |= LBM_PATH_CS_RING;
    return f;
}

lbm_status lbm_set_launch_mode(lbm_ctx* c, int32_t single_graph, int32_t pdl_direct,
                               int32_t pdl_graphs) {
    auto bit = [](int32_t v) { return v == 0 || v == 1; };
    if (!c || !bit(single_graph) || !bit(pdl_direct) || !bit(pdl_graphs)) return LBM_EINVAL;
    c->single_graph = single_graph == 1;
    c->pdl_direct = pdl_direct == 1;
    c->pdl_graph = pdl_graphs == 1;
    c->pdl_now = c->pdl_direct;
    drop_graphs(c);  // the captured launches hold the old attribute
    return LBM_OK;
}

lbm_status lbm_set_collide_form(lbm_ctx* c, int32_t ring_rows) {
    if (!c || ring_rows < -1 || ring_rows > 4096) return LBM_EINVAL;
    c->ring_rows = ring_rows;
    drop_graphs(c);  // the captured collide launches hold the old form
    return LBM_OK;
}

int64_t lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }
int64_t lbm_failed_step(const lbm_ctx* c) { return c ? c->failed : -1; }

static lbm_status init_from_device_fields(lbm_ctx* c, const double* rho, const double* ux,
                                          const double* uy) {
    c->cur = 0;
    lbm_status st = reset_state(c, 0);
    if (st) return st;
    if (is_fp64(c))
        CK(launch_init_feq<double>(rho, ux, uy, (double*)c->f[0], c->rho, c->nx, c->ny,
                                   c->plane, c->stream));
    else
        CK(launch_init_mixed(rho, ux, uy, (float*)c->f[0], c->m_rh, c->m_rl, c->nx, c->ny,
                             c->plane, c->stream));
    st = enqueue_force(c, c->stream, 0);
    if (st) return st;
    c->ready = true;
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_ctx* c, const double* h_rho, const double* h_ux,
                          const double* h_uy) {
    if (!c || !h_rho) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    st = wait_stream(c);
    if (st) return st;
    // stage in the second population buffer (>= 3 N doubles in both precisions)
    double* sg = (double*)c->f[1];
    const size_t B = c->N * sizeof(double);
    CK(cudaMemcpyAsync(sg, h_rho, B, cudaMemcpyHostToDevice, c->stream));
    if (h_ux) CK(cudaMemcpyAsync(sg + c->N, h_ux, B, cudaMemcpyHostToDevice, c->stream));
    if (h_uy) CK(cudaMemcpyAsync(sg + 2 * c->N, h_uy, B, cudaMemcpyHostToDevice, c->stream));
    st = init_from_device_fields(c, sg, h_ux ? sg + c->N : nullptr,
                                 h_uy ? sg + 2 * c->N : nullptr);
    if (st) return st;
    return read_state(c);
}

lbm_status lbm_set_fields_device(lbm_ctx* c, const double* d_rho, const double* d_ux,
                                 const double* d_uy) {
    if (!c || !d_rho) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    return init_from_device_fields(c, d_rho, d_ux, d_uy);
}

lbm_status lbm_step_async(lbm_ctx* c, int64_t n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (!c->ready) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    int64_t left = n;
    if (left >= kLongGraph) {
        st = build_graph(c, c->cur, kLongGraph, &c->graph16[c->cur]);
        if (st) return st;
        for (; left >= kLongGraph; left -= kLongGraph)
            CK(cudaGraphLaunch(c->graph16[c->cur], c->stream));
    }
    if (left >= 2) {
        st = build_graph(c, c->cur, 2, &c->graph[c->cur]);
        if (st) return st;
        for (; left >= 2; left -= 2) CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
    }
    if (left == 1) {
        if (c->single_graph) {
            st = build_graph(c, c->cur, 1, &c->graph1[c->cur]);
            if (st) return st;
            CK(cudaGraphLaunch(c->graph1[c->cur], c->stream));
        } else {
            st = enqueue_step(c, c->stream, c->cur);
            if (st) return st;
        }
        c->cur = 1 - c->cur;
    }
    c->t += n;
    return LBM_OK;
}

lbm_status lbm_check(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    return read_state(c);
}

lbm_status lbm_step(lbm_ctx* c, int64_t n) {
    lbm_status st = lbm_step_async(c, n);
    if (st) return st;
    return read_state(c);
}

lbm_status lbm_step_timed(lbm_ctx* c, float* pass_ms) {
    if (!c || !pass_ms) return LBM_EINVAL;
    if (!c->ready) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    cudaStream_t s = c->stream;
    const int from = c->cur, to = 1 - from;
    CK(cudaEventRecord(c->tev[0], s));
    st = enqueue_collide(c, s, from);
    if (st) return st;
    CK(cudaEventRecord(c->tev[1], s));
    st = enqueue_force(c, s, 1, c->tev + 2);
    if (st) return st;
    c->cur = to;
    c->t += 1;
    st = read_state(c);
    if (st) return st;
    for (int i = 0; i < 5; ++i) CK(cudaEventElapsedTime(&pass_ms[i], c->tev[i], c->tev[i + 1]));
    return LBM_OK;
}

static lbm_status fields_to_device(lbm_ctx* c, double* rho, double* vx, double* vy,
                                   double* mu) {
    const size_t B = c->N * sizeof(double);
    if (!is_fp64(c)) {
        CK(launch_macro_mixed((const float*)c->f[c->cur], c->m_rh, c->m_rl, c->m_Fx, c->m_Fy,
                              rho, vx, vy, c->nx, c->ny, c->plane, c->stream));
        if (mu) CK(launch_f_to_double<float>(c->m_dxx, mu, c->N, c->stream));  // holds mu-hat
        return LBM_OK;
    }
    if (vx || vy) {
        CK(launch_macro<double>((const double*)c->f[c->cur], c->Fx, c->Fy, vx, vy, c->nx,
                                c->ny, c->plane, c->stream));
    }
    if (rho) CK(cudaMemcpyAsync(rho, c->rho, B, cudaMemcpyDeviceToDevice, c->stream));
    if (mu) CK(cudaMemcpyAsync(mu, c->mu, B, cudaMemcpyDeviceToDevice, c->stream));
    return LBM_OK;
}

lbm_status lbm_fields_device(lbm_ctx* c, double* d_rho, double* d_vx, double* d_vy,
                             double* d_mu) {
    if (!c) return LBM_EINVAL;
    if (!c->ready) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    return fields_to_device(c, d_rho, d_vx, d_vy, d_mu);
}

lbm_status lbm_fields(lbm_ctx* c, double* h_rho, double* h_vx, double* h_vy, double* h_mu) {
    if (!c) return LBM_EINVAL;
    if (!c->ready) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    // the idle population buffer holds >= 4 N doubles in both precisions
    double* sg = staging(c);
    const size_t N = c->N;
    st = fields_to_device(c, h_rho ? sg : nullptr, h_vx ? sg + N : nullptr,
                          h_vy ? sg + 2 * N : nullptr, h_mu ? sg + 3 * N : nullptr);
    if (st) return st;
    st = wait_stream(c);
    if (st) return st;
    const size_t B = N * sizeof(double);
    if (h_rho) CK(cudaMemcpyAsync(h_rho, sg, B, cudaMemcpyDeviceToHost, c->stream));
    if (h_vx) CK(cudaMemcpyAsync(h_vx, sg + N, B, cudaMemcpyDeviceToHost, c->stream));
    if (h_vy) CK(cudaMemcpyAsync(h_vy, sg + 2 * N, B, cudaMemcpyDeviceToHost, c->stream));
    if (h_mu) CK(cudaMemcpyAsync(h_mu, sg + 3 * N, B, cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c);
}

lbm_status lbm_get_populations(lbm_ctx* c, double* h_f, int64_t* t) {
    if (!c || !h_f) return LBM_EINVAL;
    if (!c->ready) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    double* sg = staging(c);
    const size_t B = c->N * sizeof(double);
    for (int i = 0; i < 9; ++i) {
        if (is_fp64(c))
            CK(cudaMemcpyAsync(sg, (const double*)c->f[c->cur] + i * c->plane, B,
                               cudaMemcpyDeviceToDevice, c->stream));
        else
            CK(launch_f_to_double<float>((const float*)c->f[c->cur] + i * c->plane, sg, c->N,
                                         c->stream));
        st = wait_stream(c);
        if (st) return st;
        CK(cudaMemcpyAsync(h_f + i * c->N, sg, B, cudaMemcpyDeviceToHost, c->stream));
        st = wait_stream(c);
        if (st) return st;
    }
    if (t) *t = c->t;
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* h_f, int64_t t) {
    if (!c || !h_f || t < 0) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    st = wait_stream(c);
    if (st) return st;
    c->cur = 0;
    double* sg = (double*)c->f[1];
    const size_t B = c->N * sizeof(double);
    for (int i = 0; i < 9; ++i) {
        CK(cudaMemcpyAsync(sg, h_f + i * c->N, B, cudaMemcpyHostToDevice, c->stream));
        if (is_fp64(c))
            CK(cudaMemcpyAsync((double*)c->f[0] + i * c->plane, sg, B, cudaMemcpyDeviceToDevice,
                               c->stream));
        else
            CK(launch_f_from_double<float>(sg, (float*)c->f[0] + i * c->plane, c->N, c->stream));
        st = wait_stream(c);
        if (st) return st;
    }
    st = reset_state(c, t);
    if (st) return st;
    if (is_fp64(c))
        CK(launch_rho_from_f<double>((const double*)c->f[0], c->rho, c->nx, c->ny, c->plane,
                                     c->stream));
    else
        CK(launch_rho_from_f_mixed((const float*)c->f[0], c->m_rh, c->m_rl, c->nx, c->ny,
                                   c->plane, c->stream));
    st = enqueue_force(c, c->stream, 0);
    if (st) return st;
    c->ready = true;
    return read_state(c);
}

}  // extern "C"

// Body of lbm_diag with the partials buffer and its record count chosen by the
// caller (lbm_diag: the workspace's; lbm_diag_noalloc: the library's fixed array).
lbm_status cplbm_diag_with_partials(lbm_ctx* c, double* partials, int nparts, double* mass,
                                    double* max_v, double* rho_min, double* rho_max) {
    if (!c->ready) return LBM_EINVAL;
    lbm_status st = use_dev(c);
    if (st) return st;
    if (is_fp64(c))
        CK(launch_diag<double>((const double*)c->f[c->cur], c->rho, c->Fx, c->Fy, c->nx, c->ny,
                               c->plane, partials, nparts, c->dst, c->stream));
    else
        CK(launch_diag_mixed((const float*)c->f[c->cur], c->m_rh, c->m_rl, c->m_Fx, c->m_Fy,
                             c->nx, c->ny, c->plane, partials, nparts, c->dst, c->stream));
    st = read_state(c);
    if (st) return st;
    if (mass) *mass = c->hst->diag[0];
    if (max_v) *max_v = c->hst->diag[1];
    if (rho_min) *rho_min = c->hst->diag[2];
    if (rho_max) *rho_max = c->hst->diag[3];
    return LBM_OK;
}
int cplbm_ctx_device(const lbm_ctx* c) { return c->dev; }
size_t cplbm_ctx_nodes(const lbm_ctx* c) { return c->N; }

extern "C" {

lbm_status lbm_diag(lbm_ctx* c, double* mass, double* max_v, double* rho_min, double* rho_max) {
    if (!c) return LBM_EINVAL;
    return cplbm_diag_with_partials(c, c->partials, c->nparts, mass, max_v, rho_min, rho_max);
}

lbm_status lbm_cfd(const double* d_u, double* d_d1, double* d_d2, int32_t nx, int32_t ny,
                   int32_t axis, int32_t fd_order, void* cuda_stream) {
    if (!d_u || !d_d1 || nx < 1 || ny < 1 || (axis != 0 && axis != 1) ||
        (fd_order != 4 && fd_order != 6))
        return LBM_EINVAL;
    if (d_d1 == d_u || d_d2 == d_u || (d_d2 && d_d2 == d_d1)) return LBM_EINVAL;
    CK(lines_fp64_plain(d_u, d_d1, d_d2, nx, ny, axis, fd_order, (cudaStream_t)cuda_stream));
    return LBM_OK;
}

lbm_status lbm_cfd_df(const float* d_hi, const float* d_lo, float* d_d1, float* d_d2,
                      int32_t nx, int32_t ny, int32_t axis, int32_t fd_order,
                      void* cuda_stream) {
    if (!d_hi || !d_lo || !d_d1 || nx < 1 || ny < 1 || (axis != 0 && axis != 1) ||
        (fd_order != 4 && fd_order != 6))
        return LBM_EINVAL;
    const void* outs[2] = {d_d1, d_d2};
    for (const void* o : outs)
        if (o && (o == (const void*)d_hi || o == (const void*)d_lo)) return LBM_EINVAL;
    if (d_d2 == d_d1) return LBM_EINVAL;
    CK(lines_mixed_plain(d_hi, d_lo, d_d1, d_d2, nx, ny, axis, fd_order,
                         (cudaStream_t)cuda_stream));
    return LBM_OK;
}

}  // extern "C"
