// capi_batch.cu -- the batched C ABI (lbm_batch_* of include/cplbm.h): many
// independent periodic instances of the mixed path, each with its own grid and
// physical parameters, advanced together.
//
// Each instance keeps the single-instance layout (two FP32 population buffers,
// eight FP32 field planes, reduction partials) in its own region of the
// caller's workspace; a table region follows with, per pass, one argument block
// per instance and a block map (block -> instance), plus the instances' device
// state blocks side by side.  A time step is four launches for the whole batch:
//   collide-stream | x|y lines of rho | mu-hat | x|y lines of mu-hat + force
// and lbm_batch_step replays two steps as one CUDA graph.  Blocks are assigned
// to instances in decreasing order of instance size, so the long-running work
// of the large grids starts first.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "cplbm_internal.cuh"

using namespace cplbm;

namespace {

constexpr size_t kAlign = 256;
constexpr int kParts = 256;  // diagnostic partial records per instance
constexpr int kRowChoices[] = {4, 8, 16, 32};  // collide-stream strip heights

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct InstHost {
    int nx, ny;
    size_t N, plane;
    PhysParams phys;
    size_t off;  // region offset in the workspace
    float* f[2];
    float *rh, *rl, *dxr, *dyr, *dxx, *dyy, *Fx, *Fy;
    double* partials;
    int64_t t;
    bool ready;
    bool rho_df;  // density lines in double-float (else FP32), as for a lone context
    int rows;     // collide-stream strip height (0: the single-instance default)
};

struct Region {
    size_t plane, f_bytes, field_bytes, parts_off, total;
};

Region region(int nx, int ny) {
    Region r;
    r.plane = align_up((size_t)nx * ny, 64);
    r.f_bytes = align_up(9 * r.plane * sizeof(float), kAlign);
    r.field_bytes = align_up(r.plane * sizeof(float), kAlign);
    r.parts_off = 2 * r.f_bytes + 8 * r.field_bytes;
    r.total = r.parts_off + align_up(4 * kParts * sizeof(double), kAlign);
    return r;
}

// Block counts of each pass for one instance.
int cs_blocks_for(int nx, int ny, int rows) {
    return cs_mixed_blocks(cs_mixed_args(nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                         nx, ny, 0, 1.0, nullptr, nullptr, rows));
}
int mu_blocks_for(size_t N) { return (int)(((N + 3) / 4 + kMuBatchT - 1) / kMuBatchT); }

// Offsets of the table region, sized for the largest block counts (the
// smallest strip height) so that autotuning never needs more room.
struct Tables {
    size_t cs, mu, rho_df, rho_f32, force, state;
    size_t map_cs, map_mu, map_rho_df, map_rho_f32, map_force, end;
    int nb_cs, nb_mu, nb_rho_df, nb_rho_f32, nb_force;  // current counts
};

Tables table_layout(const lbm_instance* inst, int n, int order, size_t base) {
    // each density map is sized for every instance in it (the double-float
    // windows are the shorter ones, so their count bounds both kinds)
    long long cs_max = 0, mu = 0, rho = 0, force = 0;
    for (int i = 0; i < n; ++i) {
        const int nx = inst[i].grid.nx, ny = inst[i].grid.ny;
        cs_max += cs_blocks_for(nx, ny, kRowChoices[0]);
        mu += mu_blocks_for((size_t)nx * ny);
        rho += std::max(lines_batch_blocks(nx, ny, order, LineBatchKind::kRhoDF),
                        lines_batch_blocks(nx, ny, order, LineBatchKind::kRhoF32));
        force += lines_batch_blocks(nx, ny, order, LineBatchKind::kForce);
    }
    Tables t;
    size_t o = base;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, kAlign);
        return at;
    };
    t.cs = take(n * sizeof(CsBatchInst));
    t.mu = take(n * sizeof(MuBatchInst));
    t.rho_df = take(n * lines_batch_desc_bytes(LineBatchKind::kRhoDF));
    t.rho_f32 = take(n * lines_batch_desc_bytes(LineBatchKind::kRhoF32));
    t.force = take(n * lines_batch_desc_bytes(LineBatchKind::kForce));
    t.state = take(n * sizeof(DevState));
    t.map_cs = take(cs_max * sizeof(int));
    t.map_mu = take(mu * sizeof(int));
    t.map_rho_df = take(rho * sizeof(int));
    t.map_rho_f32 = take(rho * sizeof(int));
    t.map_force = take(force * sizeof(int));
    t.end = o;
    t.nb_cs = t.nb_mu = t.nb_rho_df = t.nb_rho_f32 = t.nb_force = 0;
    return t;
}

bool instance_ok(const lbm_instance& in) {
    return in.grid.nx >= 8 && in.grid.ny >= 8 && in.T_r > 0 && in.T_r < 1 && in.kappa > 0 &&
           in.tau > 0.5 && in.mesh_coeff > 0 && in.mesh_coeff <= 1 && !std::isnan(in.mu_max) &&
           (size_t)in.grid.nx * in.grid.ny <= (size_t)1 << 31;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return LBM_ECUDA;  \
    } while (0)

}  // namespace

struct lbm_batch {
    int dev, n, order;
    bool mrt;  // MRT collision (Eq. 4) for every instance
    MrtRates rates;
    cudaStream_t stream, cap_stream;
    cudaEvent_t ev, tev[5];
    char* ws;
    std::vector<InstHost> inst;
    std::vector<int> order_by_size;  // instance indices, largest grid first
    Tables tb;
    DevState* dst;  // n state blocks, device
    DevState* hst;  // pinned host mirror
    int cur;
    int line_nl;  // lines per block of the FP32 line launches (8 or 16)
    cudaGraphExec_t graph[2];
    double timeout_s;
    int failed_inst;
    int64_t failed_step;
};

namespace {

lbm_status wait_stream(lbm_batch* b) {
    CK(cudaEventRecord(b->ev, b->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaEventQuery(b->ev);
        if (q == cudaSuccess) return LBM_OK;
        if (q != cudaErrorNotReady) return LBM_ECUDA;
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > b->timeout_s) return LBM_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
    }
}

void drop_graphs(lbm_batch* b) {
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

MixedLinesView view_of(const lbm_batch* b, int i) {
    const InstHost& h = b->inst[i];
    return MixedLinesView{h.rh, h.rl, h.dxr, h.dyr, h.dxx, h.dyy, h.Fx, h.Fy, h.nx, h.ny,
                          b->dst + i};
}

// Write every pass's argument blocks and block maps to the workspace.
lbm_status upload_tables(lbm_batch* b) {
    Tables& t = b->tb;
    const int n = b->n;
    const size_t bdf = lines_batch_desc_bytes(LineBatchKind::kRhoDF);
    const size_t bf = lines_batch_desc_bytes(LineBatchKind::kRhoF32);
    const size_t bfo = lines_batch_desc_bytes(LineBatchKind::kForce);
    std::vector<CsBatchInst> cs(n);
    std::vector<MuBatchInst> mu(n);
    std::vector<unsigned char> rdf(n * bdf), rf(n * bf), force(n * bfo);
    std::vector<int> mcs, mmu, mrdf, mrf, mforce;
    for (int i : b->order_by_size) {
        const InstHost& h = b->inst[i];
        DevState* st = b->dst + i;
        CsBatchInst c;
        c.a = cs_mixed_args(h.f[0], h.f[1], h.Fx, h.Fy, h.rh, h.rl, h.nx, h.ny, h.plane,
                            h.phys.omega, b->mrt ? &b->rates : nullptr, st, h.rows);
        c.f[0] = h.f[0];
        c.f[1] = h.f[1];
        c.blk0 = (int)mcs.size();
        mcs.insert(mcs.end(), cs_mixed_blocks(c.a), i);
        cs[i] = c;

        MuBatchInst m{h.rh, h.dxx, h.dyy, h.N, mu_mixed_const(h.phys), st, (int)mmu.size()};
        mmu.insert(mmu.end(), mu_blocks_for(h.N), i);
        mu[i] = m;

        const MixedLinesView v = view_of(b, i);
        const LineBatchKind rk = h.rho_df ? LineBatchKind::kRhoDF : LineBatchKind::kRhoF32;
        std::vector<int>& mr = h.rho_df ? mrdf : mrf;
        lines_batch_fill(rk, v, b->order, (int)mr.size(),
                         h.rho_df ? rdf.data() + i * bdf : rf.data() + i * bf, b->line_nl);
        mr.insert(mr.end(), lines_batch_blocks(h.nx, h.ny, b->order, rk, b->line_nl), i);
        lines_batch_fill(LineBatchKind::kForce, v, b->order, (int)mforce.size(),
                         force.data() + i * bfo, b->line_nl);
        mforce.insert(mforce.end(),
                      lines_batch_blocks(h.nx, h.ny, b->order, LineBatchKind::kForce, b->line_nl),
                      i);
    }
    // the table region was sized for the largest counts
    const size_t cap_cs = (t.map_mu - t.map_cs) / sizeof(int);
    if (mcs.size() > cap_cs) return LBM_ENOMEM;
    t.nb_cs = (int)mcs.size();
    t.nb_mu = (int)mmu.size();
    t.nb_rho_df = (int)mrdf.size();
    t.nb_rho_f32 = (int)mrf.size();
    t.nb_force = (int)mforce.size();
    cudaStream_t s = b->stream;
    char* ws = b->ws;
    auto put = [&](size_t off, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, s)
                     : cudaSuccess;
    };
    CK(put(t.cs, cs.data(), n * sizeof(CsBatchInst)));
    CK(put(t.mu, mu.data(), n * sizeof(MuBatchInst)));
    CK(put(t.rho_df, rdf.data(), rdf.size()));
    CK(put(t.rho_f32, rf.data(), rf.size()));
    CK(put(t.force, force.data(), force.size()));
    CK(put(t.map_cs, mcs.data(), mcs.size() * sizeof(int)));
    CK(put(t.map_mu, mmu.data(), mmu.size() * sizeof(int)));
    CK(put(t.map_rho_df, mrdf.data(), mrdf.size() * sizeof(int)));
    CK(put(t.map_rho_f32, mrf.data(), mrf.size() * sizeof(int)));
    CK(put(t.map_force, mforce.data(), mforce.size() * sizeof(int)));
    // the host vectors are pageable: the copies have completed when this returns
    return wait_stream(b);
}

template <class T>
const T* at(const lbm_batch* b, size_t off) {
    return reinterpret_cast<const T*>(b->ws + off);
}

lbm_status enqueue_step(lbm_batch* b, cudaStream_t s, int from, cudaEvent_t* ev = nullptr) {
    const Tables& t = b->tb;
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    CK(launch_cs_mixed_batch(at<CsBatchInst>(b, t.cs), at<int>(b, t.map_cs), t.nb_cs, from,
                             b->mrt, s));
    CK(mark(1));
    // every instance is in exactly one of the two density launches
    CK(lines_batch_launch(LineBatchKind::kRhoF32, b->ws + t.rho_f32, at<int>(b, t.map_rho_f32),
                          t.nb_rho_f32, b->order, 1, s, b->line_nl));
    CK(lines_batch_launch(LineBatchKind::kRhoDF, b->ws + t.rho_df, at<int>(b, t.map_rho_df),
                          t.nb_rho_df, b->order, 1, s));
    CK(mark(2));
    CK(launch_mu_mixed_batch(at<MuBatchInst>(b, t.mu), at<int>(b, t.map_mu), t.nb_mu, s));
    CK(mark(3));
    CK(lines_batch_launch(LineBatchKind::kForce, b->ws + t.force, at<int>(b, t.map_force),
                          t.nb_force, b->order, 0, s, b->line_nl));
    CK(mark(4));
    return LBM_OK;
}

lbm_status build_graph(lbm_batch* b, int from) {
    if (b->graph[from]) return LBM_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    lbm_status st = enqueue_step(b, b->cap_stream, from);
    if (st == LBM_OK) st = enqueue_step(b, b->cap_stream, 1 - from);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return LBM_ECUDA;
    e = cudaGraphInstantiate(&b->graph[from], g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

// Read all state blocks back; translate the error flags.  A flagged instance
// becomes not ready (its state is undefined until it is set again) and is not
// reported again; `include` is an instance being set, checked although not ready.
lbm_status read_states(lbm_batch* b, int include = -1) {
    CK(cudaMemcpyAsync(b->hst, b->dst, b->n * sizeof(DevState), cudaMemcpyDeviceToHost,
                       b->stream));
    lbm_status w = wait_stream(b);
    if (w != LBM_OK) return w;
    int bad = -1;
    unsigned long long bad_t = ULLONG_MAX;
    for (int i = 0; i < b->n; ++i) {
        const DevState& h = b->hst[i];
        if (!h.flag || (!b->inst[i].ready && i != include)) continue;
        b->inst[i].ready = false;
        const unsigned long long ft = h.failed_t == ULLONG_MAX ? (unsigned long long)b->inst[i].t
                                                               : h.failed_t;
        if (bad < 0 || ft < bad_t) {
            bad = i;
            bad_t = ft;
        }
    }
    if (bad >= 0) {
        b->failed_inst = bad;
        b->failed_step = (int64_t)bad_t;
        return LBM_EUNSTABLE;
    }
    return LBM_OK;
}

bool all_ready(const lbm_batch* b) {
    for (const auto& h : b->inst)
        if (!h.ready) return false;
    return true;
}

lbm_status reset_state(lbm_batch* b, int i) {
    DevState h;
    std::memset(&h, 0, sizeof(h));
    h.failed_t = ULLONG_MAX;
    b->hst[i] = h;
    CK(cudaMemcpyAsync(b->dst + i, b->hst + i, sizeof(DevState), cudaMemcpyHostToDevice,
                       b->stream));
    b->inst[i].t = 0;
    return wait_stream(b);  // the pinned mirror is reused by read_states
}

// Passes 2-4 of one instance alone (its force at its current density).
lbm_status instance_force(lbm_batch* b, int i) {
    const InstHost& h = b->inst[i];
    DevState* st = b->dst + i;
    cudaStream_t s = b->stream;
    if (h.rho_df)
        CK(lines_mixed_rho_xy(h.rh, h.rl, h.dxr, h.dxx, h.dyr, h.dyy, h.nx, h.ny, b->order, st,
                              0, s));
    else
        CK(lines_mixed_rho_xy_f32(h.rh, h.dxr, h.dxx, h.dyr, h.dyy, h.nx, h.ny, b->order, st, 0,
                                  s));
    CK(launch_mu_mixed(h.rh, h.dxx, h.dyy, h.nx, h.ny, h.phys, st, s));
    CK(lines_mixed_force_xy(h.dxx, h.rh, h.dxr, h.dyr, h.Fx, h.Fy, h.nx, h.ny, b->order, s));
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(const lbm_instance* inst, int32_t n, const lbm_opts* opts) {
    if (!inst || n < 1 || !opts ||
        (opts->prec != LBM_PREC_MIXED && opts->prec != LBM_PREC_MIXED_DF) ||
        (opts->fd_order != 4 && opts->fd_order != 6))
        return 0;
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        if (!instance_ok(inst[i])) return 0;
        o += region(inst[i].grid.nx, inst[i].grid.ny).total;
    }
    return table_layout(inst, n, opts->fd_order, o).end;
}

lbm_status lbm_batch_init(lbm_batch** out, const lbm_instance* inst, int32_t n,
                          const lbm_eos* eos, const lbm_opts* opts, void* d_workspace,
                          size_t ws_bytes, void* cuda_stream) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!inst || n < 1 || !opts || !eos) return LBM_EINVAL;
    if (opts->fd_order != 4 && opts->fd_order != 6) return LBM_EINVAL;
    if (opts->prec != LBM_PREC_MIXED && opts->prec != LBM_PREC_MIXED_DF) return LBM_ENOTIMPL;
    auto rate_ok = [](double r) { return r > 0 && r < 2; };
    if (!(opts->collision == LBM_COLLIDE_BGK ||
          (opts->collision == LBM_COLLIDE_MRT && rate_ok(opts->s_e) && rate_ok(opts->s_eps) &&
           rate_ok(opts->s_q))))
        return LBM_EINVAL;
    if (!(eos->kind >= LBM_EOS_CS && eos->kind <= LBM_EOS_PR && eos->a > 0 && eos->b > 0 &&
          eos->R > 0 && std::isfinite(eos->omega)))
        return LBM_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!inst[i].grid.periodic_x || !inst[i].grid.periodic_y) return LBM_ENOTIMPL;
        if (!instance_ok(inst[i])) return LBM_EINVAL;
    }
    if (!d_workspace || ((uintptr_t)d_workspace % kAlign)) return LBM_EINVAL;
    const size_t need = lbm_batch_workspace_bytes(inst, n, opts);
    if (need == 0) return LBM_EINVAL;
    if (ws_bytes < need) return LBM_ENOMEM;
    double Tc, rc;
    if (eos_critical(eos->kind, eos->a, eos->b, eos->R, &Tc, &rc)) return LBM_EINVAL;

    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    b->n = n;
    b->order = opts->fd_order;
    b->line_nl = 8;
    b->mrt = opts->collision == LBM_COLLIDE_MRT;
    b->rates = MrtRates{opts->s_e, opts->s_eps, opts->s_q};
    b->stream = (cudaStream_t)cuda_stream;
    b->ws = (char*)d_workspace;
    b->timeout_s = 600.0;
    b->failed_inst = -1;
    b->failed_step = -1;
    b->cur = 0;
    b->graph[0] = b->graph[1] = nullptr;
    b->cap_stream = nullptr;
    b->ev = nullptr;
    for (auto& e : b->tev) e = nullptr;
    b->hst = nullptr;
    if (cudaGetDevice(&b->dev) != cudaSuccess) {
        delete b;
        return LBM_ECUDA;
    }
    b->inst.resize(n);
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        InstHost& h = b->inst[i];
        const lbm_instance& in = inst[i];
        const Region r = region(in.grid.nx, in.grid.ny);
        h.nx = in.grid.nx;
        h.ny = in.grid.ny;
        h.N = (size_t)h.nx * h.ny;
        h.plane = r.plane;
        h.off = o;
        char* base = b->ws + o;
        h.f[0] = (float*)base;
        h.f[1] = (float*)(base + r.f_bytes);
        float* fields = (float*)(base + 2 * r.f_bytes);
        const size_t fs = r.field_bytes / sizeof(float);
        float** slots[8] = {&h.rh, &h.rl, &h.dxr, &h.dyr, &h.dxx, &h.dyy, &h.Fx, &h.Fy};
        for (int q = 0; q < 8; ++q) *slots[q] = fields + q * fs;
        h.partials = (double*)(base + r.parts_off);
        PhysParams& p = h.phys;
        p.eos = eos->kind;
        p.T = in.T_r * Tc;
        p.alpha = eos_alpha(eos->kind, eos->a, eos->b, eos->R, eos->omega, p.T);
        p.a = eos->a;
        p.b = eos->b;
        p.R = eos->R;
        p.k2 = in.mesh_coeff * in.mesh_coeff;
        p.kappa = in.kappa;
        p.omega = 1.0 / in.tau;
        p.mu_cap = std::isinf(in.mu_max) ? HUGE_VAL : p.k2 * in.mu_max;
        p.cap_steps = in.mu_cap_steps;
        h.t = 0;
        h.ready = false;
        h.rows = 0;
        h.rho_df = opts->prec == LBM_PREC_MIXED_DF;
        if (!h.rho_df) {
            double rg, rl;
            h.rho_df = eos_maxwell(eos->kind, eos->a, eos->b, eos->R, eos->omega, p.T, &rg,
                                   &rl) != 0 ||
                       !(rl < kDfRatio * rg);
        }
        o += r.total;
    }
    b->tb = table_layout(inst, n, b->order, o);
    b->dst = (DevState*)(b->ws + b->tb.state);
    b->order_by_size.resize(n);
    for (int i = 0; i < n; ++i) b->order_by_size[i] = i;
    std::stable_sort(b->order_by_size.begin(), b->order_by_size.end(),
                     [&](int x, int y) { return b->inst[x].N > b->inst[y].N; });

    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&b->hst, n * sizeof(DevState)) != cudaSuccess) {
        lbm_batch_free(b);
        return LBM_ECUDA;
    }
    for (auto& e : b->tev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            lbm_batch_free(b);
            return LBM_ECUDA;
        }
    lbm_status st = LBM_OK;
    for (int i = 0; i < n && st == LBM_OK; ++i) st = reset_state(b, i);
    if (st == LBM_OK) st = upload_tables(b);
    if (st != LBM_OK) {
        lbm_batch_free(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_free(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    drop_graphs(b);
    if (b->ev) cudaEventDestroy(b->ev);
    for (auto& e : b->tev)
        if (e) cudaEventDestroy(e);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->hst) cudaFreeHost(b->hst);
    delete b;
}

lbm_status lbm_batch_set_timeout(lbm_batch* b, double seconds) {
    if (!b || !(seconds > 0)) return LBM_EINVAL;
    b->timeout_s = seconds;
    return LBM_OK;
}

int64_t lbm_batch_time(const lbm_batch* b, int32_t i) {
    if (!b || i < 0 || i >= b->n) return -1;
    return b->inst[i].t;
}

int32_t lbm_batch_tile_rows(const lbm_batch* b, int32_t i) {
    if (!b || i < 0 || i >= b->n) return -1;
    const InstHost& h = b->inst[i];
    return cs_mixed_args(nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, h.nx, h.ny, 0,
                         1.0, nullptr, nullptr, h.rows)
        .rows;
}

lbm_status lbm_batch_failed(const lbm_batch* b, int32_t* inst, int64_t* step) {
    if (!b) return LBM_EINVAL;
    if (inst) *inst = b->failed_inst;
    if (step) *step = b->failed_step;
    return LBM_OK;
}

lbm_status lbm_batch_set_fields(lbm_batch* b, int32_t i, const double* h_rho,
                                const double* h_ux, const double* h_uy) {
    if (!b || i < 0 || i >= b->n || !h_rho) return LBM_EINVAL;
    CK(cudaSetDevice(b->dev));
    lbm_status st = wait_stream(b);
    if (st) return st;
    InstHost& h = b->inst[i];
    h.ready = false;
    // stage in this instance's idle population buffer (>= 3 N doubles)
    double* sg = (double*)h.f[1 - b->cur];
    const size_t B = h.N * sizeof(double);
    CK(cudaMemcpyAsync(sg, h_rho, B, cudaMemcpyHostToDevice, b->stream));
    if (h_ux) CK(cudaMemcpyAsync(sg + h.N, h_ux, B, cudaMemcpyHostToDevice, b->stream));
    if (h_uy) CK(cudaMemcpyAsync(sg + 2 * h.N, h_uy, B, cudaMemcpyHostToDevice, b->stream));
    st = reset_state(b, i);
    if (st) return st;
    CK(launch_init_mixed(sg, h_ux ? sg + h.N : nullptr, h_uy ? sg + 2 * h.N : nullptr,
                         h.f[b->cur], h.rh, h.rl, h.nx, h.ny, h.plane, b->stream));
    st = instance_force(b, i);
    if (st) return st;
    st = read_states(b, i);
    if (st) return st;
    h.ready = true;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
    if (!b || n < 0) return LBM_EINVAL;
    if (!all_ready(b)) return LBM_EINVAL;
    CK(cudaSetDevice(b->dev));
    int64_t left = n;
    if (left >= 2) {
        lbm_status st = build_graph(b, b->cur);
        if (st) return st;
        for (; left >= 2; left -= 2) CK(cudaGraphLaunch(b->graph[b->cur], b->stream));
    }
    if (left == 1) {
        lbm_status st = enqueue_step(b, b->stream, b->cur);
        if (st) return st;
        b->cur = 1 - b->cur;
    }
    for (auto& h : b->inst) h.t += n;
    return read_states(b);
}

lbm_status lbm_batch_step_timed(lbm_batch* b, float* pass_ms) {
    if (!b || !pass_ms) return LBM_EINVAL;
    if (!all_ready(b)) return LBM_EINVAL;
    CK(cudaSetDevice(b->dev));
    CK(cudaEventRecord(b->tev[0], b->stream));
    lbm_status st = enqueue_step(b, b->stream, b->cur, b->tev);
    if (st) return st;
    b->cur = 1 - b->cur;
    for (auto& h : b->inst) h.t += 1;
    st = read_states(b);
    if (st) return st;
    for (int i = 0; i < 4; ++i) CK(cudaEventElapsedTime(&pass_ms[i], b->tev[i], b->tev[i + 1]));
    return LBM_OK;
}

lbm_status lbm_batch_fields(lbm_batch* b, int32_t i, double* h_rho, double* h_vx,
                            double* h_vy, double* h_mu) {
    if (!b || i < 0 || i >= b->n) return LBM_EINVAL;
    InstHost& h = b->inst[i];
    if (!h.ready) return LBM_EINVAL;
    CK(cudaSetDevice(b->dev));
    double* sg = (double*)h.f[1 - b->cur];  // idle buffer: >= 4 N doubles
    const size_t N = h.N;
    if (h_rho || h_vx || h_vy)
        CK(launch_macro_mixed(h.f[b->cur], h.rh, h.rl, h.Fx, h.Fy, h_rho ? sg : nullptr,
                              h_vx ? sg + N : nullptr, h_vy ? sg + 2 * N : nullptr, h.nx, h.ny,
                              h.plane, b->stream));
    if (h_mu) CK(launch_f_to_double<float>(h.dxx, sg + 3 * N, N, b->stream));  // mu-hat
    lbm_status st = wait_stream(b);
    if (st) return st;
    const size_t B = N * sizeof(double);
    if (h_rho) CK(cudaMemcpyAsync(h_rho, sg, B, cudaMemcpyDeviceToHost, b->stream));
    if (h_vx) CK(cudaMemcpyAsync(h_vx, sg + N, B, cudaMemcpyDeviceToHost, b->stream));
    if (h_vy) CK(cudaMemcpyAsync(h_vy, sg + 2 * N, B, cudaMemcpyDeviceToHost, b->stream));
    if (h_mu) CK(cudaMemcpyAsync(h_mu, sg + 3 * N, B, cudaMemcpyDeviceToHost, b->stream));
    return wait_stream(b);
}

lbm_status lbm_batch_diag(lbm_batch* b, double* mass, double* max_v, double* rho_min,
                          double* rho_max) {
    if (!b) return LBM_EINVAL;
    if (!all_ready(b)) return LBM_EINVAL;
    CK(cudaSetDevice(b->dev));
    for (int i = 0; i < b->n; ++i) {
        const InstHost& h = b->inst[i];
        CK(launch_diag_mixed(h.f[b->cur], h.rh, h.rl, h.Fx, h.Fy, h.nx, h.ny, h.plane,
                             h.partials, kParts, b->dst + i, b->stream));
    }
    lbm_status st = read_states(b);
    if (st) return st;
    for (int i = 0; i < b->n; ++i) {
        const double* d = b->hst[i].diag;
        if (mass) mass[i] = d[0];
        if (max_v) max_v[i] = d[1];
        if (rho_min) rho_min[i] = d[2];
        if (rho_max) rho_max[i] = d[3];
    }
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t reps) {
    if (!b || reps < 1) return LBM_EINVAL;
    if (!all_ready(b)) return LBM_EINVAL;
    CK(cudaSetDevice(b->dev));
    lbm_status st = wait_stream(b);
    if (st) return st;
    // one representative instance per distinct grid size
    std::map<std::pair<int, int>, int> rep;
    for (int i = 0; i < b->n; ++i) rep.emplace(std::make_pair(b->inst[i].nx, b->inst[i].ny), i);
    cudaStream_t s = b->stream;
    for (const auto& kv : rep) {
        const InstHost& h = b->inst[kv.second];
        DevState* dst = b->dst + kv.second;
        float best = 0.0f;
        int best_rows = 0;
        for (int rows : kRowChoices) {
            const CsArgs a =
                cs_mixed_args(h.f[b->cur], h.f[1 - b->cur], h.Fx, h.Fy, h.rh, h.rl, h.nx, h.ny,
                              h.plane, h.phys.omega, b->mrt ? &b->rates : nullptr, dst, rows);
            CK(launch_cs_mixed_args(a, s));  // warm-up
            CK(cudaEventRecord(b->tev[0], s));
            for (int r = 0; r < reps; ++r) CK(launch_cs_mixed_args(a, s));
            CK(cudaEventRecord(b->tev[1], s));
            st = wait_stream(b);
            if (st) return st;
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, b->tev[0], b->tev[1]));
            if (best_rows == 0 || ms < best) {
                best = ms;
                best_rows = rows;
            }
        }
        for (auto& x : b->inst)
            if (x.nx == h.nx && x.ny == h.ny) x.rows = best_rows;
    }
    // the timing launches overwrote the idle buffer and the density planes
    // with the next time level: recompute the density of the current state
    for (const auto& h : b->inst)
        CK(launch_rho_from_f_mixed(h.f[b->cur], h.rh, h.rl, h.nx, h.ny, h.plane, s));
    // lines per block of the FP32 line launches: the whole FP32 density launch
    // and the force launch of the batch, timed at 8 and 16
    {
        float best = 0.0f;
        int best_nl = 8;
        for (int nl : {8, 16}) {
            b->line_nl = nl;
            st = upload_tables(b);
            if (st) return st;
            const Tables& t = b->tb;
            auto pass = [&]() -> cudaError_t {
                cudaError_t e = lines_batch_launch(LineBatchKind::kRhoF32, b->ws + t.rho_f32,
                                                   at<int>(b, t.map_rho_f32), t.nb_rho_f32,
                                                   b->order, 0, s, nl);
                if (e != cudaSuccess) return e;
                return lines_batch_launch(LineBatchKind::kForce, b->ws + t.force,
                                          at<int>(b, t.map_force), t.nb_force, b->order, 0, s,
                                          nl);
            };
            CK(pass());  // warm-up
            CK(cudaEventRecord(b->tev[0], s));
            for (int r = 0; r < reps; ++r) CK(pass());
            CK(cudaEventRecord(b->tev[1], s));
            st = wait_stream(b);
            if (st) return st;
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, b->tev[0], b->tev[1]));
            if (nl == 8 || ms < best) {
                best = ms;
                best_nl = nl;
            }
        }
        b->line_nl = best_nl;
    }
    // the density lines overwrote mu-hat (it shares its plane with d_xx rho) and
    // the force lines then read that: recompute the force stage of the state
    for (int i = 0; i < b->n; ++i) {
        st = instance_force(b, i);
        if (st) return st;
    }
    drop_graphs(b);
    st = upload_tables(b);
    if (st) return st;
    return read_states(b);
}

int32_t lbm_batch_lines_per_block(const lbm_batch* b) { return b ? b->line_nl : -1; }

lbm_status lbm_batch_set_lines_per_block(lbm_batch* b, int32_t nl) {
    if (!b || (nl != 8 && nl != 16)) return LBM_EINVAL;
    CK(cudaSetDevice(b->dev));
    b->line_nl = nl;
    drop_graphs(b);
    return upload_tables(b);
}

}  // extern "C"
