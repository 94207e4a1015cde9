/*
 * cplbm.h -- C ABI of the GB300 (sm_103a) chemical-potential multiphase
 * lattice Boltzmann library.
 *
 * The method is that of Wen, Zhao, Qiu, Ye and Shan, "Chemical-potential
 * multiphase lattice Boltzmann method with superlarge density ratios"
 * (arXiv:1906.09530).  One time step, in the paper's notation (mesh space,
 * Sec. 4.1: grid step 1, time step 1, lattice c_s^2 = 1/3):
 *
 *   rho = sum_i f_i,  rho u = sum_i e_i f_i                           Eq. 3
 *   d_x rho, d_y rho by the compact scheme, periodic lines           Eqs. 37-39
 *   d_xx rho = D_x(D_x rho), d_yy rho = D_y(D_y rho)                 Sec. 4.3
 *   mu-hat = k^2 mu0(rho; T) - kappa-hat (d_xx rho + d_yy rho)       Eqs. 21, 33
 *   mu-hat <- min(mu-hat, k^2 mu_max) for the first mu_cap_steps     Sec. 5.6
 *   F = -rho grad(mu-hat) + c_s^2 grad(rho)                          Eq. 12
 *   F_i = f_i^eq(rho, u + F/rho) - f_i^eq(rho, u)                    Eq. 5
 *   f_i(x + e_i, t + 1) = f_i - (f_i - f_i^eq(rho, u))/tau + F_i     Eqs. 1-2
 *
 * Conventions for every call:
 *   - Fields are row-major [ny][nx] (x fastest); populations are
 *     structure-of-arrays [9][ny][nx] in the velocity order of Sec. 2:
 *     (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *   - "h_" pointers are host memory, "d_" pointers device memory of the
 *     current CUDA device.  The caller owns every pointer it passes.
 *   - Every call that can fail returns an lbm_status; LBM_OK is 0.
 *   - All device work runs on the CUDA stream given to lbm_init.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns LBM_ECUDA.
 */
#ifndef CPLBM_H
#define CPLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* an argument is out of range, or a call came out of order */
    LBM_ENOMEM = 2,    /* workspace too small, or host allocation failed */
    LBM_ECUDA = 3,     /* a CUDA runtime call failed */
    LBM_EUNSTABLE = 4, /* the device flagged rho <= 0, a non-finite value or the
                          EOS pole (b rho >= 1; b rho / 4 >= 1 for CS) while the
                          upper limit is off; see lbm_failed_step() */
    LBM_ETIMEOUT = 5,  /* device work did not finish within the wait limit */
    LBM_ENOTIMPL = 6   /* option recognised but not built (e.g. non-periodic) */
} lbm_status;

/* Equation of state (Sec. 3.2); p0 and mu0 exactly as printed:
 *   LBM_EOS_CS   Carnahan-Starling, Eqs. 20-21 (the paper: a=1, b=4, R=1)
 *   LBM_EOS_VDW  van der Waals, Eqs. 14-15 (a=9/49, b=2/21)
 *   LBM_EOS_RK   Redlich-Kwong, Eqs. 16-17 with alpha(T) = 1/sqrt(T)
 *   LBM_EOS_RKS  Soave-Redlich-Kwong, Eqs. 16-17 with alpha(T_r) of the acentric
 *                factor omega (a=2/49, b=2/21)
 *   LBM_EOS_PR   Peng-Robinson, Eqs. 18-19 with its alpha(T_r) and omega
 *                (a=2/49, b=2/21; omega 0.344 for water, 0.011 for methane) */
enum { LBM_EOS_CS = 0, LBM_EOS_VDW = 1, LBM_EOS_RK = 2, LBM_EOS_RKS = 3, LBM_EOS_PR = 4 };

/* Precision.  FP64: everything in double.  MIXED: populations and the
 * collide-stream pass in float; the density kept exactly as a double-float pair
 * (hi + lo floats); its compact-FD derivatives in float when the Maxwell density
 * ratio at T_r is below 1e4, else in double-float arithmetic wherever a line
 * window spans more than a factor 32 of density (first derivatives, rounded once
 * to float); second derivatives, chemical potential and force in float; all
 * reductions and outputs in double.  MIXED_DF: as MIXED, with the double-float
 * derivatives at every density ratio. */
enum { LBM_PREC_FP64 = 0, LBM_PREC_MIXED = 1, LBM_PREC_MIXED_DF = 2 };

typedef struct {
    int32_t nx, ny;                 /* lattice size, each >= 8 */
    int32_t periodic_x, periodic_y; /* periodic_x must be 1 (LBM_ENOTIMPL otherwise);
                                       periodic_y = 0 puts solid walls below row 0 and
                                       above row ny-1: halfway bounce-back for the
                                       populations (walls at rest unless
                                       lbm_set_wall_velocity moves them), and the
                                       density and mu-hat extended evenly about the
                                       walls for their y-derivatives (the first ghost
                                       takes its fluid neighbour's value, Sec. 5.5;
                                       d_yy rho is the compact scheme applied twice
                                       along the extended line).  Batches are
                                       periodic only. */
} lbm_grid;

typedef struct {
    int32_t kind;          /* LBM_EOS_* */
    double a, b, R, omega; /* attraction a, volume correction b, gas constant R
                              (all > 0); omega: acentric factor (RKS and PR only) */
} lbm_eos;

/* Collision.  BGK: Eq. 1 (single relaxation time tau).  MRT: Eq. 4 on the
 * standard D2Q9 moment basis (rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy),
 * S = diag(0, s_e, s_eps, 0, s_q, 0, s_q, s_v, s_v) with s_v = 1/tau; the paper
 * uses s_e = 1.64, s_eps = 1.54, s_q = 1.9.  Both with the exact-difference
 * forcing of Eq. 5. */
enum { LBM_COLLIDE_BGK = 0, LBM_COLLIDE_MRT = 1 };

typedef struct {
    int32_t prec;         /* LBM_PREC_FP64, LBM_PREC_MIXED or LBM_PREC_MIXED_DF */
    int32_t fd_order;     /* 4 (alpha = 1/4) or 6 (alpha = 1/3, Eq. 39) */
    double mu_max;        /* chemical-potential upper limit in momentum-space
                             units (Sec. 5.6); +INFINITY switches it off.  While
                             it acts, a node at or beyond the EOS pole (where mu0
                             grows without bound) gets mu-hat = k^2 mu_max */
    int64_t mu_cap_steps; /* the limit acts while the time level t < mu_cap_steps */
    int32_t collision;    /* LBM_COLLIDE_BGK (0) or LBM_COLLIDE_MRT */
    double s_e, s_eps, s_q; /* MRT rates, each in (0, 2); unused by BGK */
} lbm_opts;

/* Bytes of device workspace lbm_init needs for this grid and options, or 0
 * if the arguments are invalid.  Layout: two population buffers, the fields
 * (FP64: rho, d_x rho, d_y rho, d_xx rho, mu-hat, F_x, F_y; MIXED: rho hi, rho lo,
 * d_x rho, d_y rho, d_xx rho (then mu-hat), d_yy rho, F_x, F_y as FP32), reduction partials
 * and a small device state block, each 256-byte aligned. */
size_t lbm_workspace_bytes(const lbm_grid *grid, const lbm_opts *opts);

/* Create a simulation context.
 *   grid, eos, opts   see above (copied; the caller keeps ownership)
 *   T_r               reduced temperature T/T_c in (0, 1) (Sec. 3.2); T_c is
 *                     solved from the EOS on the host
 *   kappa             the mesh-space kappa-hat of Eq. 33, > 0
 *   tau               BGK relaxation time of Eq. 1, > 0.5
 *   mesh_coeff        the proportional coefficient k of Eq. 25, in (0, 1]
 *   d_workspace       device memory of lbm_workspace_bytes() bytes, 256-byte
 *                     aligned, owned by the caller, which must keep it alive
 *                     until lbm_free
 *   cuda_stream       a cudaStream_t (NULL = the legacy default stream); the
 *                     caller keeps ownership
 * Nothing runs on the device until lbm_set_fields.  On error *out is NULL. */
lbm_status lbm_init(lbm_ctx **out, const lbm_grid *grid, const lbm_eos *eos, double T_r,
                    double kappa, double tau, double mesh_coeff, const lbm_opts *opts,
                    void *d_workspace, size_t ws_bytes, void *cuda_stream);

/* Initial state from host FP64 fields: f_i = f_i^eq(rho, u) (Eq. 2), time
 * level 0, then the force of Eq. 12 is computed from rho.  h_ux / h_uy may be
 * NULL (zero velocity).  Returns when the device work is done. */
lbm_status lbm_set_fields(lbm_ctx *ctx, const double *h_rho, const double *h_ux,
                          const double *h_uy);

/* The same from device FP64 fields (enqueued on the stream; returns at once). */
lbm_status lbm_set_fields_device(lbm_ctx *ctx, const double *d_rho, const double *d_ux,
                                 const double *d_uy);

/* Advance n >= 0 time steps.  Steps are enqueued (in CUDA graphs of two
 * steps); the call then waits for the stream and checks the device error
 * flag.  LBM_EUNSTABLE: some step produced a bad value, lbm_failed_step()
 * names the first time level flagged, and the state is undefined until the
 * next lbm_set_fields. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Like lbm_step but returns right after enqueuing; lbm_check() later waits
 * for the stream and reads the error flag. */
lbm_status lbm_step_async(lbm_ctx *ctx, int64_t n);
lbm_status lbm_check(lbm_ctx *ctx);

/* Profiling: run one time step as direct launches (no graph) with a CUDA event
 * recorded on the stream before and after each of its passes, wait for it, and
 * return the passes' durations in milliseconds (5 slots).
 * FP64: [0] collide-stream, [1] x-lines of rho, [2] y-lines of rho + mu-hat,
 *       [3] x-lines of mu-hat + F_x, [4] y-lines of mu-hat + F_y.
 * MIXED: [0] collide-stream, [1] x- and y-lines of rho, [2] mu-hat (pointwise),
 *       [3] x- and y-lines of mu-hat + F; [4] is 0. */
lbm_status lbm_step_timed(lbm_ctx *ctx, float *pass_ms);

/* How a mixed context runs its passes (chosen at lbm_init), as a bit set:
 * LBM_PATH_RHO_DF: the density lines are double-float (density ratio at or
 *   above 1e4, or LBM_PREC_MIXED_DF), else FP32 on the hi part.
 * LBM_PATH_CS_RING: the collide-stream pass runs the row-ring kernel (see
 *   lbm_set_collide_form).
 * 0 for FP64, -1 for NULL. */
enum { LBM_PATH_RHO_DF = 2, LBM_PATH_CS_RING = 4 };
int32_t lbm_path_flags(const lbm_ctx *ctx);

/* Form of the mixed path's collide-stream pass (Eqs. 1-5 and streaming):
 *   -1  the sliding-window kernel: one warp per 30 columns, three rows of
 *       post-collision populations in registers, neighbours by warp shuffles;
 *    0  the default: the row-ring kernel on grids of at least 2^23 nodes where
 *       it applies (periodic, nx a multiple of 4 and at least 128), else the
 *       sliding window (faster on smaller grids).  A row-ring block of 128
 *       threads streams rows of 128 columns into a shared-memory ring by
 *       16-byte asynchronous copies, several rows ahead, and writes 120 of them;
 *   > 0 the row-ring kernel wherever it applies, with that many rows a block
 *       (at most 4096).
 * Both give bit-identical results; LBM_PATH_CS_RING in lbm_path_flags says
 * which one runs.  LBM_EINVAL for other values. */
lbm_status lbm_set_collide_form(lbm_ctx *ctx, int32_t ring_rows);

/* How the passes of a step are launched (results are the same either way):
 *   single_graph  1: a lone step (lbm_step_async of one step, or the odd last
 *                 step of a longer call) replays a captured one-step CUDA graph;
 *                 0: its passes are launched directly.  Longer calls always
 *                 replay graphs of 2 and 16 steps.
 *   pdl_direct, pdl_graphs  programmatic dependent launch between the kernels
 *                 of a mixed step, for direct launches and for graph-captured
 *                 ones: each kernel lets the next be scheduled once all of its
 *                 blocks have started and waits in hardware for the previous
 *                 one to complete before touching memory, so the next pass's
 *                 blocks are resident during this one's tail.
 * Defaults: single_graph 1, pdl_direct 1, pdl_graphs 0 (the fastest lone and
 * back-to-back steps measured at 1024^2).  Each argument 0 or 1, else
 * LBM_EINVAL. */
lbm_status lbm_set_launch_mode(lbm_ctx *ctx, int32_t single_graph, int32_t pdl_direct,
                               int32_t pdl_graphs);

/* Outputs of the current state to host FP64 [ny][nx] arrays, any may be NULL:
 * rho (Eq. 3), the velocity v = u + F/(2 rho) (Sec. 2, after Eq. 5) and the
 * mesh-space chemical potential mu-hat (Eq. 33).  Returns when copied. */
lbm_status lbm_fields(lbm_ctx *ctx, double *h_rho, double *h_vx, double *h_vy,
                      double *h_mu);

/* The same into device FP64 arrays (enqueued; returns at once). */
lbm_status lbm_fields_device(lbm_ctx *ctx, double *d_rho, double *d_vx, double *d_vy,
                             double *d_mu);

/* Checkpoint / resume: the populations as host FP64 [9][ny][nx] and the time
 * level.  A resume on the same build and precision is bit-exact. */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *h_f, int64_t *t);
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *h_f, int64_t t);

/* Diagnostics of the current state, FP64 reductions on the device: total mass
 * sum(rho), max |v|, min rho, max rho.  Any output may be NULL. */
lbm_status lbm_diag(lbm_ctx *ctx, double *mass, double *max_v, double *rho_min,
                    double *rho_max);

/* lbm_diag without any device allocation, for callers that cannot call
 * cudaMalloc (e.g. code whose device memory is all owned by another allocator,
 * or that may not allocate after start-up).  Same outputs as lbm_diag (FP64
 * reductions; they agree with lbm_diag to rounding of the summation order).
 * The reduction's partial sums live in a fixed 512 KB device array inside the
 * library (one 4-double record per 2048 nodes): grids above 33,554,432 nodes
 * return LBM_EINVAL.  The paper has no counterpart; this is library plumbing.
 * The first call on a device looks up that array's device address; make it
 * before any stream capture.  Like lbm_diag, every call copies its results to
 * the host and waits for the context's stream before it returns, so no call can
 * be captured into a CUDA graph: none may be made while the context's stream is
 * capturing.  Calls share the array, so calls that overlap on the GPU race on
 * it. */
lbm_status lbm_diag_noalloc(lbm_ctx *ctx, double *mass, double *max_v, double *rho_min,
                            double *rho_max);

/* Critical point (T_c, rho_c) of the EOS: the point where dp0/drho and
 * d2p0/drho2 both vanish (Sec. 3.2).  Host only. */
lbm_status lbm_critical(const lbm_eos *eos, double *Tc, double *rhoc);

/* Maxwell equal-area coexistence densities at reduced temperature T_r: equal
 * pressure and equal chemical potential on the two stable branches (Sec. 5.1).
 * Host only. */
lbm_status lbm_maxwell(const lbm_eos *eos, double T_r, double *rho_g, double *rho_l);

/* Stand-alone compact-FD derivative of a device FP64 field [ny][nx] along
 * axis 0 (x) or 1 (y), periodic, Eqs. 37-38 with alpha = 1/4 (fd_order 4) or
 * 1/3 (fd_order 6, Eq. 39).  d_d1 receives D u; d_d2, if not NULL, receives
 * D(D u) ("applying CFM twice", Sec. 4.3).  The outputs must not overlap the
 * input.  Enqueued on cuda_stream; returns at once. */
lbm_status lbm_cfd(const double *d_u, double *d_d1, double *d_d2, int32_t nx, int32_t ny,
                   int32_t axis, int32_t fd_order, void *cuda_stream);

/* The mixed path's line solve, stand-alone: derivative along axis 0 (x) or 1 (y)
 * of a periodic field given as an unevaluated double-float sum hi + lo of two
 * device FP32 arrays [ny][nx] (the form the mixed path keeps the density in).
 * d_d1 receives D u computed in double-float arithmetic and rounded to FP32;
 * d_d2, if not NULL, receives D(D u) computed in FP32 (Eqs. 37-39, Sec. 4.3).
 * Outputs must not overlap the inputs.  Enqueued on cuda_stream. */
lbm_status lbm_cfd_df(const float *d_hi, const float *d_lo, float *d_d1, float *d_d2,
                      int32_t nx, int32_t ny, int32_t axis, int32_t fd_order,
                      void *cuda_stream);

/* Time level of the current state, and the first flagged time level after
 * LBM_EUNSTABLE (-1 if none). */
int64_t lbm_time(const lbm_ctx *ctx);
int64_t lbm_failed_step(const lbm_ctx *ctx);

/* Host wait limit, in seconds, for lbm_step / lbm_check / copies (default 600). */
lbm_status lbm_set_timeout(lbm_ctx *ctx, double seconds);

/* Walls moving along x, as seen from a moving reference frame (Sec. 5.5):
 * u_bottom, u_top are the x-velocities of the wall below row 0 and above row
 * ny-1, lattice units.  The population reflected at a wall moving at U gains
 * -2 w_i rho (e_i . U) / c_s^2 (Ladd's moving-wall bounce-back), rho the node's
 * own density; mass is conserved.  Takes effect from the next step.
 * LBM_EINVAL if the grid has no walls or |u| >= 0.5. */
lbm_status lbm_set_wall_velocity(lbm_ctx *ctx, double u_bottom, double u_top);

/* ---- Batches: many independent instances advanced together -------------
 *
 * A batch holds n periodic instances of the MIXED path, each with its own grid,
 * T_r, kappa-hat, tau, k and upper limit, and one EOS and one fd_order.  Every
 * time step runs the four passes of the mixed path once for the whole batch
 * (one launch per pass, blocks mapped to instances), two steps per CUDA graph,
 * so small instances do not each pay for their own launches.  Within one
 * instance the arithmetic is that of a single lbm_ctx with the same arguments:
 * a batch member and a lone context give bit-identical results.
 *
 * Workspace: one device buffer owned by the caller (256-byte aligned,
 * lbm_batch_workspace_bytes long): the instances' populations and fields, their
 * device state blocks, the per-instance argument tables and block maps.  It must
 * outlive the batch.  Host arrays are [ny][nx] FP64 of the instance's own grid.
 */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

typedef struct {
    lbm_grid grid;         /* nx, ny >= 8, periodic in both directions */
    double T_r;            /* T / T_c in (0, 1) */
    double kappa;          /* kappa-hat > 0 (Eq. 33, mesh space) */
    double tau;            /* relaxation time > 0.5 (Eq. 1) */
    double mesh_coeff;     /* k in (0, 1] (Eq. 25) */
    double mu_max;         /* upper limit, momentum-space units (Sec. 5.6); +INFINITY: off */
    int64_t mu_cap_steps;  /* the limit acts while the instance's time level < this */
} lbm_instance;

/* Bytes of device workspace for the batch (0 if an argument is invalid).
 * opts->prec must be LBM_PREC_MIXED or LBM_PREC_MIXED_DF (chosen per instance by
 * its density ratio, as for a lone context); opts->mu_max / mu_cap_steps are unused
 * (each instance carries its own). */
size_t lbm_batch_workspace_bytes(const lbm_instance *inst, int32_t n, const lbm_opts *opts);

/* Create a batch of n >= 1 instances on the current CUDA device.  LBM_EINVAL for
 * an out-of-range instance, LBM_ENOTIMPL for walls, another EOS or FP64, and
 * LBM_ENOMEM if ws_bytes is too small.  Copies the argument tables to the
 * workspace and returns when they are there. */
lbm_status lbm_batch_init(lbm_batch **out, const lbm_instance *inst, int32_t n,
                          const lbm_eos *eos, const lbm_opts *opts, void *d_workspace,
                          size_t ws_bytes, void *cuda_stream);

/* Initial state of instance i: f = f^eq(rho, u) with u = 0 where ux / uy are NULL;
 * its force is computed at once and its time level set to 0.  Every instance
 * must be set before the first step.  Returns when done; LBM_EUNSTABLE if the
 * input itself is flagged (instance i stays unset). */
lbm_status lbm_batch_set_fields(lbm_batch *b, int32_t i, const double *h_rho,
                                const double *h_ux, const double *h_uy);

/* Advance every instance by n >= 0 time steps and check the device error flags.
 * LBM_EUNSTABLE: an instance flagged rho <= 0, a non-finite value or the EOS
 * pole (see lbm_batch_failed); that instance's state is undefined and it must be
 * set again before the next step, the others are valid.  LBM_EINVAL if any
 * instance has not been set. */
lbm_status lbm_batch_step(lbm_batch *b, int64_t n);

/* One step with CUDA events around each pass; pass_ms[0..3] receive the times
 * of collide-stream, the x|y lines of rho, mu-hat and the x|y lines of mu-hat
 * with the force, each over the whole batch (milliseconds). */
lbm_status lbm_batch_step_timed(lbm_batch *b, float *pass_ms);

/* Outputs of instance i as in lbm_fields (any pointer may be NULL). */
lbm_status lbm_batch_fields(lbm_batch *b, int32_t i, double *h_rho, double *h_vx,
                            double *h_vy, double *h_mu);

/* Per-instance diagnostics into host arrays of n doubles (any may be NULL):
 * mass, max |v|, min rho, max rho. */
lbm_status lbm_batch_diag(lbm_batch *b, double *mass, double *max_v, double *rho_min,
                          double *rho_max);

/* Time the collide-stream pass of one instance of each distinct grid size for
 * each strip height the kernel supports (reps launches each, CUDA events), keep
 * the fastest for every instance of that size, and rebuild the batch's tables.
 * The simulation state is left as it was.  Returns when done. */
lbm_status lbm_batch_autotune(lbm_batch *b, int32_t reps);

/* The strip height in use for instance i (rows of the collide-stream warps). */
int32_t lbm_batch_tile_rows(const lbm_batch *b, int32_t i);

/* Lines per block (8 or 16) of the batch's FP32 line launches: the density
 * lines of the instances below the double-float ratio, and every instance's
 * force lines (lbm_batch_autotune times both and keeps the faster; the
 * double-float density lines always take 8).  Results do not depend on it.
 * The getter returns -1 for NULL; the setter LBM_EINVAL for other values. */
int32_t lbm_batch_lines_per_block(const lbm_batch *b);
lbm_status lbm_batch_set_lines_per_block(lbm_batch *b, int32_t nl);

/* Time level of instance i (-1 if out of range). */
int64_t lbm_batch_time(const lbm_batch *b, int32_t i);

/* After LBM_EUNSTABLE: the first flagged instance (smallest flagged time level,
 * then smallest index) and its flagged time level; -1 / -1 if none. */
lbm_status lbm_batch_failed(const lbm_batch *b, int32_t *inst, int64_t *step);

/* Host wait limit, in seconds (default 600). */
lbm_status lbm_batch_set_timeout(lbm_batch *b, double seconds);

/* Release the batch (not the workspace or the stream). */
void lbm_batch_free(lbm_batch *b);

/* ---- The surrogate network of the warm start ------------------------------
 *
 * A multilayer perceptron 4 -> 256 -> 256 -> 256 -> 256 (tanh on the three hidden
 * layers, linear output) that maps (T_r, kappa-hat, k, 1/R), scaled by the
 * caller, to a 256-point equilibrium interface profile (R the radius of a drop;
 * the caller's scaling of 1/R is constant for flat interfaces).  Every matrix product runs on the
 * tensor cores in BF16 with FP32 accumulation; master weights, Adam moments,
 * activations and the gradient are FP32.  The products are tcgen05 MMAs with
 * the accumulator in tensor memory (the weight gradient split over the batch
 * and its partials added in a fixed order, so results do not depend on timing);
 * an mma.sync kernel is kept as the comparison point.  A tcgen05 product whose
 * bounded wait runs out sets an error word that the next call that waits for
 * the stream (set/get_params, a loss read) reports as LBM_ETIMEOUT.  Loss: mean squared error over the
 * batch and the 256 outputs.  Training: Adam (beta1 0.9, beta2 0.999, eps 1e-8,
 * with bias correction).  The parameters are one flat FP32 vector in the order
 * W1, b1, W2, b2, W3, b3, W4, b4, each W row-major [fan_in][fan_out].
 *
 * Workspace: one caller-owned device buffer (256-byte aligned,
 * lbm_mlp_workspace_bytes(max_batch) long).  Inputs d_x are device FP32
 * [batch][4], targets and outputs device FP32 [batch][256], 1 <= batch <=
 * max_batch.  All work is enqueued on the stream given to lbm_mlp_init. */
typedef struct lbm_mlp lbm_mlp; /* opaque, owned by the library */

int64_t lbm_mlp_param_count(void); /* 198 656 */
size_t lbm_mlp_workspace_bytes(int32_t max_batch); /* 0 if max_batch is out of range */
lbm_status lbm_mlp_init(lbm_mlp **out, int32_t max_batch, void *d_workspace, size_t ws_bytes,
                        void *cuda_stream);
/* Set the parameters from a host vector (and reset Adam's moments and step
 * count); returns when copied. */
lbm_status lbm_mlp_set_params(lbm_mlp *net, const float *h_params);
/* Copy the parameters into a host vector of lbm_mlp_param_count() floats;
 * returns when copied. */
lbm_status lbm_mlp_get_params(lbm_mlp *net, float *h_params);
/* y = network(x), enqueued. */
lbm_status lbm_mlp_forward(lbm_mlp *net, const float *d_x, int32_t batch, float *d_y);
/* The loss of (x, t) and its gradient with respect to every parameter (into
 * d_grad, a device FP32 vector of lbm_mlp_param_count() entries; NULL: kept
 * inside).  h_loss, if not NULL, receives the loss and makes the call wait. */
lbm_status lbm_mlp_loss_grad(lbm_mlp *net, const float *d_x, const float *d_t, int32_t batch,
                             double *h_loss, float *d_grad);
/* One Adam step with learning rate lr > 0 on the batch (x, t). */
lbm_status lbm_mlp_train_step(lbm_mlp *net, const float *d_x, const float *d_t, int32_t batch,
                              float lr, double *h_loss);
/* Product path: 1 = tcgen05 (the default), 0 = the mma.sync tile kernel (kept
 * as the comparison point).  LBM_EINVAL for other values. */
lbm_status lbm_mlp_set_tcgen05(lbm_mlp *net, int32_t on);
/* 1 while the products run on tcgen05; 0 when switched off, or after a tensor
 * map could not be made (the library then falls back to mma.sync); -1 for NULL. */
int32_t lbm_mlp_tcgen05(const lbm_mlp *net);
/* Release the network (not the workspace or the stream); NULL is a no-op. */
void lbm_mlp_free(lbm_mlp *net);

/* A static, NUL-terminated description of a status; never NULL (unknown codes
 * get a generic message). */
const char *lbm_strerror(lbm_status s);

/* Release the context (not the workspace or the stream, which the caller owns). */
void lbm_free(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CPLBM_H */
