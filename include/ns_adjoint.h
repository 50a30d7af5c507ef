/*
 * ns_adjoint.h - C ABI of the GB300 (sm_103a) unsteady discrete adjoint of the
 * compressible Navier-Stokes equations (Talnikar, Wang & Laskowski, arXiv 1511.06959).
 *
 * Problem statement (section "Unsteady adjoint"): march w_t + div(F - F^v) = s
 * (Eq. e:vector) forward in time, accumulate the time-averaged pressure-loss objective
 * Jbar (Eq. e:pressure_loss), then integrate the adjoint backward from a zero terminal
 * condition, recomputing primal states from checkpoints ("Implementation").  The
 * stabilised adjoint adds div(lambda sigma_1 grad w_hat) where sigma_1 is the largest
 * singular value of the growth matrix M = M1 - M2 ("Energy analysis").
 *
 * Discretisation: periodic structured box of nx*ny*nz cells (nz = 1 is a 2D box),
 * central 2nd-order face fluxes (optionally with the paper's Roe dissipation,
 * ns_params.flux), compact viscous stencil, classical RK4 or the paper's SSP-RK3
 * (ns_params.scheme) with a constant dt; the adjoint is the exact transpose of that
 * discrete map.
 *
 * Conventions shared by every call:
 *  - Field pointers are DEVICE pointers owned by the caller, in SoA layout
 *    [batch][5][nz][ny][nx] (x fastest), components (rho, rho u1, rho u2, rho u3, rho E)
 *    for states and the same order for adjoints.  Scalar fields (sigma_1, nu) are
 *    [batch][nz][ny][nx].  All must be 8-byte aligned (cudaMalloc memory is).
 *    HOST memory appears only where a call says so: the plan (ns_plan), the energy fit
 *    and the choice of lambda (ns_energy_efolds, ns_lambda_select, the candidate and
 *    report arrays of ns_estimate_lambda), the snapshot arena of NS_CKPT_STRIDE_HOST
 *    (ns_run_opts.host_arena), the parameter structs, and values a call returns.  The
 *    snapshot file of NS_CKPT_STRIDE_DISK (ns_run_opts.disk_path) is the one file the
 *    library writes.
 *  - Work is enqueued on the stream given to ns_create (or ns_set_stream) and is
 *    asynchronous unless a call says it returns a host value.
 *  - Every call returns NS_OK (0) or a negative NS_ERR_* code.  NS_ERR_ARG: null
 *    context, null required pointer, bad size, or an aliasing rule broken.
 *    NS_ERR_BUDGET: a caller-provided buffer (arena, host arena, work buffer, plan
 *    array) is smaller than the call needs; these size checks run before the call
 *    enqueues any work.
 *    NS_ERR_CUDA: a launch or allocation failed.  NS_ERR_IO: a snapshot file access
 *    of NS_CKPT_STRIDE_DISK failed.  Faults found on the device
 *    (non-finite values, an unstable adjoint viscosity) set a sticky error word
 *    that ns_last_error() reads back.
 *  - A context owns only its workspace (stage buffers and reduction scratch,
 *    allocated by ns_create), never the caller's fields.  One context must not be
 *    used from two host threads at once.
 */
#ifndef NS_ADJOINT_H
#define NS_ADJOINT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NS_OK 0
#define NS_ERR_ARG (-1)
#define NS_ERR_BUDGET (-2)
#define NS_ERR_NONFINITE (-3)
#define NS_ERR_UNSTABLE (-4)
#define NS_ERR_CUDA (-5)
#define NS_ERR_CORRUPT (-6) /* a verified checkpoint snapshot changed between store and load */
#define NS_ERR_BOUNDS (-7)  /* bounds-checking builds only (NS_DEBUG_BOUNDS): a stencil kernel
                               met a field index outside its field and skipped the access */
#define NS_ERR_IO (-8)      /* NS_CKPT_STRIDE_DISK: the snapshot file could not be created,
                               written or read (the sweep stops; errno is left as set) */

/* time integration (ns_params.scheme) */
#define NS_RK4 0    /* classical four-stage fourth-order Runge-Kutta, constant dt */
#define NS_SSPRK3 1 /* three-stage third-order strong-stability-preserving Runge-Kutta
                       (section "Numerical methods"; Shu-Osher form
                       W2 = w + dt R(w), W3 = 3/4 w + 1/4 (W2 + dt R(W2)),
                       w' = 1/3 w + 2/3 (W3 + dt R(W3))) */

/* convective face flux (ns_params.flux) */
#define NS_FLUX_CENTRAL 0 /* Phi = (F_L + F_R)/2 - F^v */
#define NS_FLUX_ROE 1     /* the approximate Roe solver of section "Numerical methods":
                             Phi = (F_L + F_R)/2 - |A~|(w_R - w_L)/2 - F^v, with A~ the Roe
                             matrix (sqrt(rho)-weighted Roe state) and Harten's entropy fix */

#define NS_FP64 0  /* every flux, transpose and stage state in FP64 */
#define NS_MIXED 1 /* fluxes, transposes and stage states in FP32; w, adjoint, objective,
                      reductions and time accumulation in FP64 */

typedef struct {
  int nx, ny, nz;   /* cells per direction; nz = 1 is a 2D box */
  int batch;        /* independent boxes, leading dimension of every field */
  double dx, dy, dz;/* cell sizes */
  double gamma;     /* ratio of specific heats (1.4), Eq. (e:navier) */
  double mu;        /* constant dynamic viscosity, Eq. (e:navier) */
  double Pr;        /* Prandtl number (0.72); heat flux alpha = gamma mu / Pr */
  double dt;        /* constant time step */
  int precision;    /* NS_FP64 or NS_MIXED */
  int plane_i;      /* objective plane = x-face between cell columns plane_i-1, plane_i
                       (taken modulo nx; must lie within (-2^30, 2^30)) */
  double pt_in;     /* reference stagnation pressure p_t,in of Eq. (e:pressure_loss) */
  int scheme;       /* NS_RK4 or NS_SSPRK3: the explicit Runge-Kutta method of every step,
                       its tangent and its discrete adjoint */
  int flux;         /* NS_FLUX_CENTRAL or NS_FLUX_ROE (convective face flux) */
  double roe_delta; /* NS_FLUX_ROE: Harten's entropy fix, |lam| -> (lam^2 + delta^2)/(2 delta)
                       where |lam| < delta = roe_delta * (Roe-averaged sound speed); > 0 */
} ns_params;

typedef struct ns_ctx ns_ctx;

/* Create a context: validates params, allocates the workspace (5 stage-state fields
 * of the precision's stage type plus reduction scratch) on the current device.
 * stream: a cudaStream_t (NULL = default stream). */
int ns_create(const ns_params* p, void* stream, ns_ctx** out);
void ns_destroy(ns_ctx* ctx);
int ns_set_stream(ns_ctx* ctx, void* stream);
int ns_set_dt(ns_ctx* ctx, double dt);
/* Bytes of device workspace this context holds. */
size_t ns_workspace_bytes(const ns_ctx* ctx);

/* R = R(w) + s: the semi-discrete right-hand side (Eq. e:vector with source s,
 * section "Unsteady adjoint").  s may be NULL.  R must not alias w. */
int ns_rhs(ns_ctx* ctx, const double* w, const double* s, double* R);

/* Rd = (dR/dw)(w) wd: the tangent of the residual (test support for the
 * dot-product identity).  FP64 in both precision modes. */
int ns_rhs_tangent(ns_ctx* ctx, const double* w, const double* wd, double* Rd);

/* out = (dR/dw)(w)^T a + L_nu a: the transposed residual Jacobian, the discrete form
 * of the A_kji, A^v_kji and D_kjil terms of the adjoint equation (section "Unsteady
 * adjoint"), plus the added adjoint viscosity div(nu grad a) when nu != NULL
 * (section "Energy analysis", stabilised adjoint).  out must not alias w or a. */
int ns_rhs_transpose(ns_ctx* ctx, const double* w, const double* a, const float* nu,
                     double* out);

/* w_out = one step (RK4 or SSP-RK3, ns_params.scheme) of w_in with source s (may be
 * NULL).  w_out must not alias w_in. */
int ns_primal_step(ns_ctx* ctx, const double* w_in, const double* s, double* w_out);

/* Tangent of one step (FP64): wd_out = d(w^{n+1})/d(w^n) wd_in + d/ds sd.
 * s is the primal source (may be NULL), sd its perturbation (may be NULL). */
int ns_tangent_step(ns_ctx* ctx, const double* w_n, const double* s, const double* wd_in,
                    const double* sd, double* wd_out);

/* Discrete adjoint of one step ("Implementation": the adjoint of the discrete
 * scheme, with the primal stage states recomputed from w_n):
 *   lam_n = (d w^{n+1} / d w^n)^T lam_np1
 * nu: per-cell added adjoint viscosity (NULL = none), applied in each of the stage
 *     products.
 * sbar_acc: if not NULL, sbar_acc += sum of the stage seeds; the source
 *     sensitivity dJ/ds of a time-constant source is the final sbar_acc.
 * lam_n must not alias lam_np1 or w_n. */
int ns_adjoint_step(ns_ctx* ctx, const double* w_n, const double* s, const double* lam_np1,
                    const float* nu, double* lam_n, double* sbar_acc);
/* ns_adjoint_step with an FP64 viscosity field nu (double [batch][nz][ny][nx], may be
 * NULL); FP64 contexts only (NS_ERR_ARG in MIXED).  With ns_growth_sigma1_f64 and
 * ns_add_adjoint_viscosity_f64 the stabilised adjoint step ("Energy analysis") runs with
 * every operand in FP64. */
int ns_adjoint_step_f64(ns_ctx* ctx, const double* w_n, const double* s, const double* lam_np1,
                        const double* nu, double* lam_n, double* sbar);

/* Pressure loss on the plane (Eq. e:pressure_loss, instantaneous plane average):
 *   J_acc[b] += weight * J(w_b)  for each box b (device array of batch doubles),
 *   lam += weight * dJ/dw        if lam != NULL (only the two plane columns change).
 * FP64 in both modes; a non-finite J sets NS_ERR_NONFINITE. */
int ns_objective(ns_ctx* ctx, const double* w, double weight, double* J_acc, double* lam);

/* sigma_1 per cell: the largest singular value of M = M1 - M2 built from central
 * differences of rho, u, p, a, b (section "Energy analysis", closed forms of M1 and M2;
 * for nz = 1 the (rho, u1, u2, p) block).  stats (device, may be NULL) receives
 * [batch][2] = (max, mean) per box. */
int ns_growth_sigma1(ns_ctx* ctx, const double* w, float* sigma1, double* stats);
/* ns_growth_sigma1 with sigma_1 kept in FP64 (sigma1: double [batch][nz][ny][nx]); FP64
 * contexts only (NS_ERR_ARG in MIXED).  Section "Energy analysis" defines sigma_1; the
 * FP64 form lets the stabilised adjoint of an FP64 context keep every operand in FP64. */
int ns_growth_sigma1_f64(ns_ctx* ctx, const double* w, double* sigma1, double* stats);

/* nu = lambda * sigma_1 where sigma_1 > tau, else 0 (section "Energy analysis":
 * the lambda sigma_1 coefficient; tau = 0 is the paper's rule).  lambda has units of
 * length^2.  If dt * nu * sum_d 4/dx_d^2 exceeds the scheme's real-axis stability limit
 * (2.78 for RK4, 2.51 for SSP-RK3) in any cell, NS_ERR_UNSTABLE is set in the sticky
 * error word. */
int ns_add_adjoint_viscosity(ns_ctx* ctx, const float* sigma1, double lambda, double tau,
                             float* nu);
/* The same rule in FP64: nu = lambda sigma_1 where sigma_1 > tau, else 0 (double fields),
 * with the same stability check (NS_ERR_UNSTABLE in the sticky error word). */
int ns_add_adjoint_viscosity_f64(ns_ctx* ctx, const double* sigma1, double lambda, double tau, double* nu);

/* Separate added-viscosity factors for the adjoints of rho, of rho u (three
 * components) and of rho E: every later use of nu by this context (adjoint steps, the
 * transposed residual, ns_apply_adjoint_viscosity, sweeps, the stability check of
 * ns_add_adjoint_viscosity, which uses the largest factor) multiplies the viscosity term
 * of each component by its factor.  The conclusion names different adjoint viscosities
 * for the different state variables as a next step; (1, 1, 1), the default, is the
 * single coefficient of section "Energy analysis".  split: host array of 3 finite
 * non-negative values, else NS_ERR_ARG. */
int ns_set_viscosity_split(ns_ctx* ctx, const double* split);

/* cap != 0: every added adjoint viscosity this context forms afterwards (the sigma_1 rule
 * of ns_add_adjoint_viscosity(_f64) and of the sweeps, and the learned closure) is held
 * at the explicit stability limit named above in the cells where it would exceed it,
 * instead of being left there and flagged with NS_ERR_UNSTABLE; a non-finite value is
 * still flagged.  cap = 0 (the default) restores the flag. */
int ns_set_viscosity_cap(ns_ctx* ctx, int cap);

/* out += L_nu a = div(nu grad a) per component, nu_face = mean of the two cells
 * (the discrete added-viscosity operator alone), times the component's factor of
 * ns_set_viscosity_split. */
int ns_apply_adjoint_viscosity(ns_ctx* ctx, const float* nu, const double* a, double* out);

/* Adjoint energy E[b] = sum_cells v_hat . v_hat dV with w_hat = T^T v_hat, T = S V
 * (section "Symmetrization"; "Energy analysis" defines E_vhat).  E: device array of
 * batch doubles, overwritten.  A non-finite value sets NS_ERR_NONFINITE. */
int ns_adjoint_energy(ns_ctx* ctx, const double* w, const double* lam, double* E);

/* out[m] = <a, phi_m> for m < nphi over n elements (FP64, deterministic).
 * phi is [nphi][n]; out is a device array of nphi doubles, overwritten. */
int ns_dot(ns_ctx* ctx, const double* a, const double* phi, int nphi, size_t n, double* out);

/* s = sum_m theta[m] phi_m over n elements (device theta[nphi], phi[nphi][n]). */
int ns_combine(ns_ctx* ctx, const double* theta, const double* phi, int nphi, size_t n,
               double* s);

/* out[i] = in[i] rounded to binary32 (nearest, ties to even) for n elements, on the
 * context's stream; results below the smallest normal float flush to signed zero.
 * This is the conversion the mixed-precision path uses for its float mirrors. */
int ns_to_float(ns_ctx* ctx, const double* in, float* out, size_t n);

/* max over all cells of |u| + c; writes one double to the device pointer out. */
int ns_max_wave_speed(ns_ctx* ctx, const double* w, double* out);

/* ------------------------------------------------------------------------------
 * Checkpointed adjoint sweep ("Implementation": periodic snapshots of the primal,
 * segments recomputed during the backward sweep).  The host runtime plans which
 * primal states to keep (ns_plan) and executes the plan on the context's stream
 * (ns_adjoint_run).  Schedules:
 *   NS_CKPT_ALL     keep every state (no recomputation)
 *   NS_CKPT_STRIDE  keep every param-th state; replay one segment at a time and keep
 *                   all its states during its reversal.  The last segment is not
 *                   replayed: the forward pass keeps its states, so a sweep advances
 *                   nsteps + ((nsteps - 1) / param) * (param - 1) primal steps.  With two
 *                   or more segments (and verify off, on a periodic box) the sweep is
 *                   pipelined: the replay of the next segment runs on a second stream
 *                   while the current one is reversed, with a second set of segment
 *                   states and kept stages in the arena; the bits are those of the
 *                   sequential order.  ns_set_pipeline turns this off.
 *   NS_CKPT_REVOLVE binomial checkpointing with param state slots: each step is
 *                   recomputed at most r times, r the least integer with
 *                   C(param + r, param) >= nsteps
 *   NS_CKPT_STRIDE_HOST  NS_CKPT_STRIDE with the every-param-th snapshots in host
 *                   memory (a caller-owned host arena, ns_run_opts.host_arena): each
 *                   snapshot is copied out once in the forward pass and back once when
 *                   its segment is replayed; only the replayed segment's states live
 *                   in device memory (and, from the forward pass, the last segment's,
 *                   which is not replayed).  Pipelined like NS_CKPT_STRIDE (each replay
 *                   copies its snapshot back on the replay stream); ns_set_pipeline(ctx, 0)
 *                   keeps the device footprint smallest.  The copies run on the context's stream, so a
 *                   sweep gives the same bits as NS_CKPT_STRIDE.  On a Grace-hosted GPU
 *                   they cross NVLink-C2C.
 *   NS_CKPT_STRIDE_DISK  the plan of NS_CKPT_STRIDE_HOST with the snapshots in a file
 *                   (ns_run_opts.disk_path) instead of host memory: each snapshot is
 *                   written once in the forward pass and read once when its segment is
 *                   replayed, through a page-locked staging buffer of one state that the
 *                   library allocates.  The stream is drained around each file access, so
 *                   the sweep waits for the file system; it gives the same bits as
 *                   NS_CKPT_STRIDE.  The file is created (truncated) by the forward pass,
 *                   is written only by the library while the sweep holds it, and is
 *                   removed when the sweep is released.  Use it for horizons whose
 *                   snapshots fit neither device nor host memory.
 *   NS_CKPT_REVOLVE_HOST, NS_CKPT_REVOLVE_DISK  the binomial plan of NS_CKPT_REVOLVE with
 *                   its param checkpoint slots in host memory (ns_run_opts.host_arena,
 *                   ns_run_host_bytes) or in a file (ns_run_opts.disk_path): every store
 *                   and load of a checkpoint becomes a copy out or back, and the device
 *                   holds only the two working states.  The same bits as NS_CKPT_REVOLVE;
 *                   the slot count, and with it the recomputation, is then bounded by host
 *                   memory or disk instead of HBM.
 * ---------------------------------------------------------------------------- */
#define NS_CKPT_ALL 0
#define NS_CKPT_STRIDE 1
#define NS_CKPT_REVOLVE 2
#define NS_CKPT_STRIDE_HOST 3
#define NS_CKPT_STRIDE_DISK 4
#define NS_CKPT_REVOLVE_HOST 5
#define NS_CKPT_REVOLVE_DISK 6

#define NS_OP_ADVANCE 1 /* advance the current state from step a to step b */
#define NS_OP_STORE 2   /* keep the current state (step a) in slot b */
#define NS_OP_LOAD 3    /* make the state of step a in slot b current (b = -1: w^0) */
#define NS_OP_ADJOINT 4 /* reverse step a (current state is w^a), then add the
                           objective source of step a if a >= 1 */
#define NS_OP_FREE 5    /* release slot b (held step a) */
#define NS_OP_SOURCE 6  /* add the objective source of step a (current state w^a) */
#define NS_OP_STORE_HOST 7 /* copy the current state (step a) to host slot b (the file's
                              slot b for NS_CKPT_STRIDE_DISK) */
#define NS_OP_LOAD_HOST 8  /* copy the state of step a from host (file) slot b into a free
                              device buffer and make it current */
#define NS_OP_FREE_HOST 9  /* release host (file) slot b (held step a) */

typedef struct {
  int op, a, b;
} ns_action;

/* Plan a sweep of nsteps steps (pure host computation, no CUDA call).  Writes up to
 * max_actions actions to out (out may be NULL to query the count), the number of
 * actions to *n_actions, the largest number of simultaneously used device slots to
 * *slots_used (host slots are not counted: see ns_run_host_bytes) and the number of
 * primal steps advanced (first pass included) to *advances.  NS_ERR_ARG for nsteps < 1, a bad schedule or param < 1 where needed;
 * NS_ERR_BUDGET if max_actions is too small (n_actions still reports the need). */
int ns_plan(int nsteps, int schedule, int param, ns_action* out, int max_actions, int* n_actions,
            int* slots_used, long long* advances);

typedef struct {
  int nsteps;        /* primal steps N; Jbar = (1/N) sum_{n=1..N} J(w^n) */
  int schedule;      /* NS_CKPT_* */
  int param;         /* stride (NS_CKPT_STRIDE, NS_CKPT_STRIDE_HOST, NS_CKPT_STRIDE_DISK) or
                        state slots (NS_CKPT_REVOLVE, NS_CKPT_REVOLVE_HOST, NS_CKPT_REVOLVE_DISK) */
  double lambda;     /* added adjoint viscosity nu = lambda sigma_1 [sigma_1 > tau]; 0 = none */
  double tau;
  int record_energy; /* write E_vhat(w^n, lam^n), n = 0..N, to energy[n][batch] */
  int record_sigma;  /* write (max, mean) of sigma_1(w^n), n = 0..N-1, to sigma_stats[n][batch][2]
                        (sigma_1 is always evaluated when lambda > 0) */
  const void* mlp;   /* learned closure (device network blob, see ns_mlp_*), or NULL: when set,
                        nu = lambda dx^2 sigma_1 softplus(MLP(f)) replaces the sigma_1 rule
                        (lambda is then the global factor kappa) */
  void* host_arena;  /* NS_CKPT_STRIDE_HOST, NS_CKPT_REVOLVE_HOST: caller-owned host memory of at least
                        ns_run_host_bytes bytes for the snapshots (page-locked, e.g.
                        cudaHostAlloc, for the copies to run asynchronously; pageable
                        memory works but each copy then blocks the host); else ignored.
                        The host must not touch it while a sweep runs. */
  size_t host_bytes; /* its size in bytes */
  int verify;        /* nonzero: a 64-bit checksum of every stored snapshot (device slots and
                        host slots) is taken when it is stored and checked when it is loaded;
                        a mismatch sets NS_ERR_CORRUPT in the sticky error word.  The
                        checksum sums, mod 2^64, a 64-bit mix (the splitmix64 finaliser) of
                        each 64-bit word keyed by its position, so any changed, lost or
                        moved word changes it except with probability 2^-64, and its
                        parallel sum is exact in any order.  Costs one read of the state
                        per store and per load. */
  const char* disk_path; /* NS_CKPT_STRIDE_DISK, NS_CKPT_REVOLVE_DISK: path of the snapshot file (NS_ERR_ARG if
                        NULL); else ignored.  The string is copied by the forward pass. */
} ns_run_opts;

/* Device bytes the caller must provide as the arena of ns_adjoint_run (state slots,
 * two working states, one adjoint field, sigma_1 and nu fields, scalars; for a stride
 * plan one segment's kept stage states and mirrors, and when the sweep is pipelined a
 * second set of them with param - 1 segment states per set, see ns_set_pipeline). */
size_t ns_run_arena_bytes(const ns_ctx* ctx, const ns_run_opts* o);

/* Host bytes of the snapshot arena of an NS_CKPT_STRIDE_HOST or NS_CKPT_REVOLVE_HOST sweep
 * (one FP64 state per snapshot held at once); 0 for the other schedules or a NULL
 * argument. */
size_t ns_run_host_bytes(const ns_ctx* ctx, const ns_run_opts* o);

/* Whole forward + checkpointed backward sweep from w^0 with the time-constant source s
 * (may be NULL): Jbar[batch] (device) receives the time-averaged pressure loss,
 * lam0 (device field) dJbar/dw^0, sbar (device field, may be NULL) dJbar/ds.
 * energy / sigma_stats: device arrays or NULL (see ns_run_opts).  arena: caller-owned
 * device memory of at least ns_run_arena_bytes(ctx, o) bytes, 256-byte aligned;
 * NS_ERR_BUDGET if it is smaller, or if an NS_CKPT_STRIDE_HOST sweep's host_arena is
 * NULL or shorter than ns_run_host_bytes(ctx, o).  The sweep is deterministic: replayed
 * states are bitwise identical to the first pass. */
int ns_adjoint_run(ns_ctx* ctx, const double* w0, const double* s, const ns_run_opts* o,
                   void* arena, size_t arena_bytes, double* Jbar, double* lam0, double* sbar,
                   double* energy, double* sigma_stats);

/* The two halves of ns_adjoint_run, for callers that separate the forward pass from the
 * reverse sweep (an autograd wrapper).  ns_forward_run executes the plan up to the
 * objective source at step N: it keeps the planned checkpoints in the arena and
 * accumulates Jbar.  ns_backward_run then reverses the sweep on the same context and
 * arena (w0, s and the arena must be unchanged in between) with a unit seed on Jbar:
 * lam0 = dJbar/dw^0, sbar = dJbar/ds (may be NULL), energy / sigma_stats as in
 * ns_adjoint_run.  A forward run is reversed at most once; NS_ERR_ARG otherwise. */
int ns_forward_run(ns_ctx* ctx, const double* w0, const double* s, const ns_run_opts* o,
                   void* arena, size_t arena_bytes, double* Jbar);
int ns_backward_run(ns_ctx* ctx, double* lam0, double* sbar, double* energy, double* sigma_stats);
/* Generation of the forward sweep that awaits its ns_backward_run: every successful
 * ns_forward_run numbers its sweep 1, 2, ... on this context; 0 when no forward sweep is
 * pending (none ran, it was reversed, or a later forward replaced it).  A caller that
 * keeps several losses of one context (an autograd graph) records the number after its
 * forward and compares it before its backward, so that it never reverses another
 * forward's trajectory.  The paper has no counterpart. */
long long ns_sweep_generation(const ns_ctx* ctx);

/* Pipelined stride sweeps on this context (NS_CKPT_STRIDE above): on = 1 (the default
 * unless the environment sets NS_PIPELINE=0) or 0.  The pipelined arena holds a second
 * set of param - 1 segment states and of kept stages (ns_run_arena_bytes follows the
 * setting); its replays run on a context the library creates on first use with this
 * context's parameters, which reports into this context's error word.  NS_ERR_ARG for a
 * NULL context. */
int ns_set_pipeline(ns_ctx* ctx, int on);

/* ------------------------------------------------------------------------------
 * A whole sweep as one CUDA graph.  ns_adjoint_run_capture records the launches,
 * copies and stream forks of one ns_adjoint_run call with these arguments into a CUDA
 * graph instead of running them; ns_graph_launch replays them on the context's stream
 * as one graph launch.  A replay does all of the sweep's work again (forward pass,
 * replays, adjoint steps, diagnostics): it reads w0 and s as they are at replay time and
 * overwrites Jbar, lam0, sbar, energy and sigma_stats, and gives the same bits as
 * ns_adjoint_run on the same inputs.  It keeps the pointers, the ns_run_opts values and
 * the context's settings (dt, viscosity split and cap, boundaries, learned closure
 * parameters' location) of the capture: the caller captures again after changing any of
 * them.  The arena and the output arrays belong to the graph while it is replayed.
 * Capture runs on a stream the library owns, so it works whatever stream the context
 * uses.  NS_ERR_ARG for the host and disk tiers (their copies go through the host) and
 * for a NULL out; the errors of ns_adjoint_run otherwise; NS_ERR_CUDA if the CUDA
 * runtime refuses the capture.  The paper has no counterpart: this is how the sweep's
 * thousands of short launches are issued from one host call. */
typedef struct ns_graph ns_graph;
int ns_adjoint_run_capture(ns_ctx* ctx, const double* w0, const double* s, const ns_run_opts* o,
                           void* arena, size_t arena_bytes, double* Jbar, double* lam0, double* sbar,
                           double* energy, double* sigma_stats, ns_graph** out);
/* One replay on the context's current stream (ns_set_stream), ordered after the work
 * already on it.  NS_ERR_ARG for a NULL graph. */
int ns_graph_launch(ns_graph* graph);
/* Kernel launches of one replay (this library's kernels; ns_launch_count does not count
 * replays); -1 for a NULL graph. */
long long ns_graph_kernels(const ns_graph* graph);
/* Releases the graph (NULL is ignored).  The caller synchronises its replays first. */
void ns_graph_destroy(ns_graph* graph);

/* ------------------------------------------------------------------------------
 * Choice of the viscosity scaling factor lambda for a given problem.  The paper's
 * conclusion names this as the method's first open question; its results section
 * tabulates adjoint against finite-difference sensitivity over lambda: too little
 * viscosity leaves the adjoint growing, too much biases the sensitivity, and in between
 * the sensitivity hardly moves with lambda.  The rule below (the smallest candidate
 * that damps the adjoint energy and sits on that plateau) is a reading of the table and
 * of section "Energy analysis", not a procedure the paper states.
 * ---------------------------------------------------------------------------- */

/* Growth of the adjoint energy over the second half of the backward sweep beyond what
 * the objective source alone accounts for, in e-folds, per box (pure host computation,
 * no CUDA call).  E: host array [nsteps+1][batch] of E_vhat(w^m, lam^m) as
 * ns_adjoint_run records it; out: host array [batch].  lam^m sums the sources of steps
 * m..N (N - m + 1 bounded terms), so with a propagator that does not expand the energy
 * sqrt(E^m) grows at most linearly in N - m + 1 and E^m / (N - m + 1)^2 stays bounded.
 * With M = nsteps / 2 (integer division), out[b] = -M times the least-squares slope of
 * ln(E[m][b] / (N - m + 1)^2) against m over m = 0..M: the fitted rise across the window
 * as the adjoint runs backward from step M to step 0 (about 0 or below for a damped
 * adjoint, a M for one growing like exp(a (N - m))).  A non-positive or non-finite
 * energy in the window gives +infinity for that box.  NS_ERR_ARG for nsteps < 2,
 * batch < 1 or a NULL pointer. */
int ns_energy_efolds(const double* E, int nsteps, int batch, double* out);

/* Index of the smallest candidate i < n - 1 with efolds[i] <= efold_tol and
 * change[i] <= rel_tol, else -1 (pure host computation).  efolds: host array [n];
 * change: host array [n - 1]; candidates in ascending lambda.  -1 also for n < 2 or a
 * NULL array; NaN entries never qualify. */
int ns_lambda_select(int n, const double* efolds, const double* change, double efold_tol, double rel_tol);

/* Device bytes of the work buffer of ns_estimate_lambda: three fields (lam0 and two
 * source sensitivities), the energy series [nsteps+1][batch], Jbar[batch] and two
 * norms, each 256-byte aligned.  0 for a NULL argument. */
size_t ns_estimate_work_bytes(const ns_ctx* ctx, const ns_run_opts* o);

/* Runs ns_adjoint_run with the options o, o->lambda replaced by each of the n
 * candidates lambdas[0] < ... < lambdas[n-1] (host array, all >= 0), the energy series
 * recorded and no sigma_1 statistics, and reports on the host:
 *   efolds[i]  max over boxes of ns_energy_efolds of candidate i's energy series;
 *   change[i]  (i < n - 1) ||sbar_{i+1} - sbar_i|| / ||sbar_{i+1}||, the relative L2
 *              change over all boxes and components of the source sensitivity dJbar/ds
 *              from candidate i to candidate i + 1 (norms in FP64 on the device; 0 when
 *              both norms are 0, +infinity when only ||sbar_{i+1}|| is);
 *   *chosen    ns_lambda_select(n, efolds, change, efold_tol, rel_tol).
 * With o->mlp set the candidates are values of the closure's global factor kappa.
 * w0, s (may be NULL): as in ns_adjoint_run; arena: as in ns_adjoint_run for o (its
 * size does not depend on lambda).  work: device memory of at least
 * ns_estimate_work_bytes(ctx, o) bytes, 256-byte aligned.  Synchronises the context's
 * stream after each candidate (the host reads the energy series and the norms).
 * NS_ERR_ARG for n < 2, candidates not strictly ascending or negative, nsteps < 2 or a
 * NULL pointer (s excepted); NS_ERR_BUDGET for a short arena or work buffer; errors of
 * ns_adjoint_run are passed through, with the reports of the candidates before the
 * failing one filled in. */
int ns_estimate_lambda(ns_ctx* ctx, const double* w0, const double* s, const ns_run_opts* o,
                       const double* lambdas, int n, double efold_tol, double rel_tol, void* arena,
                       size_t arena_bytes, void* work, size_t work_bytes, double* efolds, double* change,
                       int* chosen);

/* field[b] *= seed[b] for every box b of a [batch][5][cells] field (device seed[batch]):
 * applies a per-box output cotangent to unit-seed adjoints. */
int ns_scale_boxes(ns_ctx* ctx, const double* seed, double* field);

/* out[m] = sum_b sum_cells field[b][comp][cell] * phi[m][cell] for m < nphi (FP64,
 * deterministic): the gradient of a time-constant source s[b][comp] = sum_m theta_m phi_m
 * shared by all boxes, from the source sensitivity field. */
int ns_dot_boxes(ns_ctx* ctx, const double* field, int comp, const double* phi, int nphi,
                 double* out);

/* Kernel timing for roofline reports: when on, the context records a CUDA event pair
 * around the consecutive adjoint-stage launches of each adjoint step (4 for RK4, 3 for
 * SSP-RK3; the time between them is the launches and the in-stream gaps between them);
 * ns_profile_read synchronises and returns the summed milliseconds of the pairs and the
 * number of adjoint-stage launches they bracket since profiling was enabled. */
int ns_profile_enable(ns_ctx* ctx, int on);
int ns_profile_read(ns_ctx* ctx, double* ms, long long* launches);

/* ns_objective without any device allocation.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc, such as host frameworks that own every byte
 * of device memory through their own pool or quota, or timing loops that must not take
 * cudaMalloc's implicit device synchronisation.  It needs no context: p describes the
 * grid, stream is a cudaStream_t (NULL = default stream) that must belong to the
 * current device (else NS_ERR_ARG).  It computes what ns_objective computes
 * (J_acc[b] += weight * J(w_b); lam += weight * dJ/dw if lam != NULL), equal to it to FP64
 * roundoff, with the three-kernel form of the objective (per-block partial sums, a final
 * reduction, the gradient scatter) instead of ns_objective's two kernels; its reduction
 * scratch is a file-scope device array of 256 KiB held by every GPU that loads the
 * library until the process exits.
 *  - Limit: batch <= 55 (2 * 296 * batch + 2 * batch doubles must fit); larger batches
 *    return NS_ERR_BUDGET before any work is enqueued.  The size limits of ns_create
 *    apply; plane_i is taken modulo nx, as in ns_objective, and must lie within
 *    (-2^30, 2^30).
 *  - The first call on a device looks up the array's device address on that device
 *    (cudaGetSymbolAddress, with that device current); make that first call before
 *    any stream capture.  NS_ERR_CUDA if the lookup fails.
 *  - All calls share the one array: calls that overlap on the GPU (different streams,
 *    no ordering between them) race and give wrong results.
 *  - There is no sticky error word: a non-finite J simply shows in J_acc. */
int ns_objective_noalloc(const ns_params* p, void* stream, const double* w, double weight,
                         double* J_acc, double* lam);

/* ------------------------------------------------------------------------------
 * Learned adjoint-viscosity closure.  The paper tunes one constant lambda by hand in
 * the stabilised adjoint (section "Energy analysis") and leaves its automatic estimation
 * open (conclusion); here a per-cell coefficient is predicted from local flow features:
 *   nu(x) = kappa dx^2 sigma_1(x) softplus(MLP(f(x))),
 * MLP 14 -> 64 -> 64 -> 1 with GELU hidden layers, BF16 weights on the tensor cores,
 * FP32 accumulation.  Features f: the symmetrised variables S(q_bar)(q - q_bar) about the
 * box-mean primitive state, over the mean sound speed, and the 9 central-difference
 * entries of grad u times L / c_bar (L = 1); stored as 16 floats per cell (last two 0).
 * A network is a caller-owned device blob of ns_mlp_net_bytes() bytes holding FP32
 * master parameters (NS_MLP_PARAMS, order W1[14][64], b1[64], W2[64][64], b2[64],
 * w3[64], b3), the Adam moments and the inference copies.
 * ---------------------------------------------------------------------------- */
#define NS_MLP_PARAMS 5185
size_t ns_mlp_net_bytes(void);
/* master parameters = params (device, NS_MLP_PARAMS floats), Adam moments zeroed */
int ns_mlp_set_params(ns_ctx* ctx, void* net, const float* params);
/* params (device, NS_MLP_PARAMS floats) = the FP32 master parameters */
int ns_mlp_get_params(ns_ctx* ctx, const void* net, float* params);
/* out (device, NS_MLP_PARAMS floats) = the first (which = 1) or second (which = 2) Adam
 * moment of the network */
int ns_mlp_get_moment(ns_ctx* ctx, const void* net, int which, float* out);
/* feat[batch * cells][16] from w */
int ns_mlp_features(ns_ctx* ctx, const double* w, float* feat);
/* nu = kappa dx^2 sigma_1 softplus(MLP(feat)) for every cell; NS_ERR_UNSTABLE is set in
 * the sticky error word as for ns_add_adjoint_viscosity */
int ns_mlp_infer(ns_ctx* ctx, const void* net, const float* feat, const float* sigma1, double kappa,
                 float* nu);
/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8; step >= 1 counts from 1) on the mean
 * squared error of softplus(MLP(feat[idx[i]])) against target[idx[i]], i < n, with the
 * forward pass quantised exactly as ns_mlp_infer.  loss (device float, may be NULL)
 * receives the minibatch loss before the update.  The first call, or a larger n,
 * allocates the context's training scratch. */
int ns_mlp_train_step(ns_ctx* ctx, void* net, const float* feat, const float* target, const int* idx,
                      int n, int step, double lr, float* loss);
/* Training label: acc[cell] += max(0, v_hat^T M v_hat) / |grad v_hat|^2 with
 * w_hat = lam, v_hat = T^-T w_hat ("Symmetrization") and M the growth matrix of
 * Eq. (e:energy_1): the viscosity that balances local growth and the dissipation of an
 * identity-Laplacian added term.  2D boxes use the (rho, u1, u2, p) block. */
int ns_adjoint_label(ns_ctx* ctx, const double* w, const double* lam, float* acc);
/* Training target t = min(acc / (dx^2 sigma_1), t_max) per cell (the label as a
 * coefficient of dx^2 sigma_1, the form the network predicts) */
int ns_label_target(ns_ctx* ctx, const float* acc, const float* sigma1, double t_max, float* target);

/* Synchronises the stream, then returns and clears the sticky device error word
 * (NS_OK, NS_ERR_NONFINITE or NS_ERR_UNSTABLE). */
int ns_last_error(ns_ctx* ctx);
const char* ns_error_string(int code);

/* ------------------------------------------------------------------------------
 * Bounded boxes: characteristic (non-reflecting) inflow at x = 0 and outflow at
 * x = L_x (section "Numerical methods": non-reflecting inlet and outlet; section
 * "Energy analysis": the incoming characteristics are set there) and isothermal
 * no-slip walls at y = 0 and y = L_y (the vane surface is isothermal, section "Problem
 * setup"); z stays periodic.  The paper gives no discrete form; here each boundary has
 * one ghost layer:
 *  - inflow/outflow ghost columns hold the boundary state of the x-direction Riemann
 *    invariants R+- = u1 +- 2c/(gamma-1): at the outflow R+, the entropy p/rho^gamma
 *    and the tangential velocity from the adjacent cell and R- from the far field; at
 *    the inflow R- from the adjacent cell and the rest from the far field;
 *  - wall ghost rows hold the adjacent cell's density, its momentum reversed and the
 *    internal energy 2 e_w - e (zero face velocity, the wall's face temperature),
 *    built over the ghost columns, so a corner is the wall's ghost of the inflow or
 *    outflow ghost.
 * The residual is the periodic residual of the padded box, cropped; the adjoint is its
 * exact transpose (the ghosts' Jacobians pulled back); the added adjoint viscosity
 * passes no flux through boundary faces; sigma_1 uses the ghosts.  Fields stay
 * unpadded [batch][5][nz][ny][nx]: the context pads and crops internally.
 * ---------------------------------------------------------------------------- */
#define NS_BC_PERIODIC 0
#define NS_BC_INOUT 1        /* characteristic inflow and outflow in x */
#define NS_BC_WALLS 2        /* isothermal no-slip walls in y */
#define NS_BC_INOUT_WALLS 3  /* both */
/* Set the boundaries of a context.  far: the far-field primitive state (rho, u1, u2, u3,
 * p) of the characteristic conditions (rho, p > 0; needed with inflow/outflow);
 * wall_e: the internal energy e = c_v T of the bottom and the top wall (> 0; needed
 * with walls).  Allocates the padded workspace (NS_ERR_CUDA on failure); synchronises
 * the context's stream.  On a bounded context ns_rhs, ns_rhs_transpose,
 * ns_primal_step, ns_adjoint_step(_f64), ns_growth_sigma1(_f64) (stats NULL),
 * ns_objective (a plane inside the box), ns_add_adjoint_viscosity(_f64),
 * ns_adjoint_energy and ns_max_wave_speed apply, and so do the checkpointed sweeps
 * (ns_adjoint_run, ns_forward_run / ns_backward_run, ns_estimate_lambda): they run the
 * step calls above on every action of their plan, the states recomputed inside each
 * adjoint step, with the same bits as those calls made step by step; a bounded sweep
 * takes neither sigma_1 statistics (record_sigma) nor the learned closure (mlp), which
 * are NS_ERR_ARG.  The tangent calls, ns_apply_adjoint_viscosity, the closure's
 * features and label and slab groups return NS_ERR_ARG.  NS_BC_PERIODIC restores the
 * periodic box. */
int ns_set_boundaries(ns_ctx* ctx, int bc, const double* far, const double* wall_e);

/* ------------------------------------------------------------------------------
 * x-slab decomposition (section "Numerical methods": the paper's solver splits its
 * domain over MPI ranks).  A box of NX columns is cut into slabs along x; slab k is
 * held by its own context as a padded box of nx_k = (its interior columns) + 2 cells in
 * x: columns 0 and nx_k - 1 are ghost columns that hold the neighbouring slabs'
 * boundary columns, and the slabs are periodic as a whole (slab 0's left neighbour is
 * the last slab).  With ghosts current, every call of a context on its padded slab
 * (residual, transpose, sigma_1, ...) gives the unsplit box's values in the interior
 * columns, because the discrete residual and its transpose reach one cell in x; the
 * group calls below run the Runge-Kutta stages of all slabs in turn and exchange each
 * stage's output field between them, so that the interior columns of a step or an
 * adjoint step equal the unsplit box's bit for bit.  Ghost-column values of outputs
 * are those of the neighbours after each call.  Reductions are per slab: a slab's
 * objective needs the plane's two columns in its interior, and sums over slabs (J, the
 * adjoint energy) are the caller's (for several processes an allreduce).
 * ---------------------------------------------------------------------------- */
typedef struct ns_slab_group ns_slab_group;
/* Host exchange of one slab's ghost columns for a group of one slab per process:
 * field is the slab's device field [batch][ncomp][nz][ny][nx] of elem_bytes-byte
 * values; the function fills columns 0 and nx-1 from the neighbouring processes' columns
 * nx-2 (left neighbour) and 1 (right neighbour) in stream order on the slab context's
 * stream and returns 0, or nonzero on failure. */
typedef int (*ns_halo_exchange_fn)(void* user, void* field, int elem_bytes, int ncomp);
/* slabs: n contexts, left to right, on padded slabs (nx >= 3) with the same ny, nz,
 * batch, precision, scheme, flux, cell sizes, dt and fluid constants (else NS_ERR_ARG).
 * Each may have its own stream (and device): exchanges order the streams with events.
 * The group keeps the context pointers; destroy it before its contexts. */
int ns_slab_group_create(ns_ctx* const* slabs, int n, ns_slab_group** out);
void ns_slab_group_destroy(ns_slab_group* group);
/* Replace the in-process exchange (one strided device copy per ghost column) with a
 * host function, for a group of exactly one slab whose neighbours live in other
 * processes (NS_ERR_ARG otherwise); fn = NULL restores the in-process exchange. */
int ns_slab_set_exchange(ns_slab_group* group, ns_halo_exchange_fn fn, void* user);
/* Fill the ghost columns of fields[k] (device, slab k, elem_bytes 4 or 8, ncomp
 * components) from the neighbouring slabs. */
int ns_slab_exchange(ns_slab_group* group, void* const* fields, int elem_bytes, int ncomp);
/* One step (ns_primal_step) of every slab: w[k] -> wo[k], s NULL or one source per
 * slab; w's ghost columns must be current; wo's are current on return. */
int ns_slab_primal_step(ns_slab_group* group, const double* const* w, const double* const* s,
                        double* const* wo);
/* One adjoint step (ns_adjoint_step without sbar) of every slab: lam[k] -> lo[k]; w,
 * lam and nu (NULL, or one float field per slab) must have current ghost columns; lo's
 * are current on return. */
int ns_slab_adjoint_step(ns_slab_group* group, const double* const* w, const double* const* s,
                         const double* const* lam, const float* const* nu, double* const* lo);
/* Workspace bytes of ns_slab_adjoint_run for each slab (bytes[k], host array of n). */
int ns_slab_run_bytes(ns_slab_group* group, const ns_run_opts* o, size_t* bytes);
/* The checkpointed sweep of ns_adjoint_run on a slab group: the same plan (NS_CKPT_ALL,
 * NS_CKPT_STRIDE or NS_CKPT_REVOLVE; the host and disk tiers are NS_ERR_ARG) executed on
 * every slab, each slab's states kept in its own workspace (work[k], device, 256-byte
 * aligned, at least ns_slab_run_bytes; NS_ERR_BUDGET otherwise).  Slab `own` holds the
 * objective plane (its two columns interior to it): it evaluates J and its source and
 * Jbar (device, batch doubles, on own's stream) receives J-bar; lam0[k] (device fields)
 * receives dJ-bar/dw^0 of each slab with current ghost columns.  With o->lambda > 0 the
 * sigma_1 rule's viscosity is formed per slab (float, as ns_slab_adjoint_step takes it)
 * and its ghost columns exchanged.  The learned closure, the energy and sigma_1 series,
 * snapshot checksums (verify) and a source sensitivity are not available here
 * (NS_ERR_ARG).  The results equal the same slab calls made step by step. */
int ns_slab_adjoint_run(ns_slab_group* group, int own, const double* const* w0, const double* const* s,
                        const ns_run_opts* o, void* const* work, const size_t* work_bytes, double* Jbar,
                        double* const* lam0);

/* Measured arithmetic peak of the current device: the rate of independent fused
 * multiply-adds (2 flops each) of kind NS_PEAK_FP32 (scalar FFMA), NS_PEAK_FP32X2 (the
 * paired FP32 instruction) or NS_PEAK_FP64, in flop/s, from CUDA events around a
 * full-occupancy kernel of about 20 ms (best of several launches).  The paper has no
 * counterpart: the stencil kernels here are bound by FP32 arithmetic and instruction
 * issue, and this is the denominator of their arithmetic roofline fraction.  Allocates
 * and frees a small device buffer, a stream and two events; synchronises; NS_ERR_CUDA if
 * a launch fails. */
#define NS_PEAK_FP32 0
#define NS_PEAK_FP32X2 1
#define NS_PEAK_FP64 2
int ns_measure_fma_peak(int kind, double* flops_per_s);

/* Number of CUDA kernels this library has launched in this process, over all contexts
 * (monotone; host-side count, no device synchronisation).  The paper has no
 * counterpart: it lets a caller state how many kernels a region of its own launched. */
unsigned long long ns_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* NS_ADJOINT_H */
