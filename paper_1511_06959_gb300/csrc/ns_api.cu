// C-ABI entry points (include/ns_adjoint.h): argument checks, workspace ownership and
// the sequencing of the fused stage kernels into Runge-Kutta (RK4, SSP-RK3) primal,
// tangent and adjoint steps.
#include <cuda_runtime.h>

#include <cmath>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "../../include/ns_adjoint.h"
#include "ns_common.cuh"
#include "ns_kernels.h"
#include "ns_ctx.h"
#include "ns_mlp.h"

using ns::Coef;
using ns::Dual;
using ns::GridDesc;

namespace {

template <class T>
Coef<T> make_coef(const ns_params& p) {
  Coef<T> c;
  c.gamma = T(p.gamma);
  c.gm1 = T(p.gamma - 1.0);
  c.mu = T(p.mu);
  c.alpha = T(p.gamma * p.mu / p.Pr);
  c.roe_delta = T(p.roe_delta);
  c.roe = p.flux == NS_FLUX_ROE ? 1 : 0;
  const double d[3] = {p.dx, p.dy, p.dz};
  for (int i = 0; i < 3; ++i) {
    c.idx[i] = T(1.0 / d[i]);
    c.i4dx[i] = T(0.25 / d[i]);
    c.hidx[i] = T(0.5 / d[i]);
  }
  return c;
}

int cuerr(cudaError_t e) { return e == cudaSuccess ? NS_OK : NS_ERR_CUDA; }


bool mixed(const ns_ctx* c) { return c->p.precision == NS_MIXED; }

}  // namespace

enum { WF = 0, LF = 1, W2 = 2, W3 = 3, W4 = 4, AA = 5, AB = 6, GS = 7, SB = 8 };

template <class T>
static T* buf(ns_ctx* c, int i) {
  return (T*)c->stage[i];
}

static int ensure_tangent_buffers(ns_ctx* c) {
  for (int i = 0; i < 6; ++i) {
    if (!c->tan[i]) {
      if (cudaMalloc(&c->tan[i], c->field * sizeof(double)) != cudaSuccess) return NS_ERR_CUDA;
      c->ws_bytes += c->field * sizeof(double);
    }
  }
  return NS_OK;
}

// Explicit Runge-Kutta tableaux in the increment-sum form the stage kernels use.  Stage
// i (0-based) evaluates k_i = R(W_i), adds dt b_i k_i to the increment sum D, and forms
// the next stage state W_{i+1} = w + dt cout_i k_i + cd_i D.  The adjoint runs the stages
// backwards (launch j = 0 is the last stage): the seed of the last stage is dt ca0 lam,
// and launch j < ns-1 forms the seed of the stage before it as
// dt (cl_j lam + cg_j g + cs_j G), G the sum of the products g of the launches so far
// (the transpose of a_{i+1,i} g_{i+1} + sum_{m>i+1} a_{m,i} g_m).  limit: the step's
// stability interval on the negative real axis (for the added adjoint viscosity).
struct Scheme {
  int ns;
  double b[4], cout[4], cd[4];
  double ca0, cl[3], cg[3], cs[3];
  double limit;
  bool needs_sum() const { return cd[0] != 0 || cd[1] != 0 || cd[2] != 0 || cd[3] != 0; }
};

// classical RK4: W2 = w + dt/2 k1, W3 = w + dt/2 k2, W4 = w + dt k3, b = (1,2,2,1)/6
static const Scheme kRK4 = {4,
                            {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6},
                            {0.5, 0.5, 1.0, 0.0},
                            {0, 0, 0, 0},
                            1.0 / 6,
                            {1.0 / 3, 1.0 / 3, 1.0 / 6},
                            {1.0, 0.5, 0.5},
                            {0, 0, 0},
                            2.78};
// SSP-RK3 (section "Numerical methods"): the Shu-Osher stages in tableau form,
// W2 = w + dt k1, W3 = w + dt/4 (k1 + k2) = w + 3/2 D, b = (1, 1, 4)/6; adjoint seeds
// a3 = 2/3 dt lam, a2 = dt (lam/6 + g3/4), a1 = dt (lam/6 + g2 + g3/4)
static const Scheme kSSPRK3 = {3,
                               {1.0 / 6, 1.0 / 6, 2.0 / 3, 0},
                               {1.0, 0.0, 0.0, 0.0},
                               {0, 1.5, 0, 0},
                               2.0 / 3,
                               {1.0 / 6, 1.0 / 6, 0},
                               {0.25, 0.75, 0},
                               {0, 0.25, 0},
                               2.51};

static const Scheme& scheme_of(const ns_ctx* c) { return c->p.scheme == NS_SSPRK3 ? kSSPRK3 : kRK4; }

// One step with the increment sum D in the stage type and one FP64 add
// w^{n+1} = w^n + D at the last stage.  keep (may be null): buffers that receive the
// stage states W2..W_ns of this step; wo_mirror (may be null): receives w^{n+1} rounded
// to the stage type.
template <class CT>
static int primal_step_t(ns_ctx* c, const Coef<CT>& cf, const CT* W1, const double* w, const double* s,
                         double* wo, CT* wo_mirror = nullptr, CT* const* keep = nullptr) {
  const Scheme& sc = scheme_of(c);
  const double dt = c->p.dt;
  CT* D = buf<CT>(c, GS);
  const CT* in = W1;
  for (int i = 0; i < sc.ns; ++i) {
    const bool last = i == sc.ns - 1;
    CT* out = last ? nullptr : (keep ? keep[i] : buf<CT>(c, i % 2 == 0 ? W2 : W3));
    ns::StageArgs<CT, CT> a{};
    a.W = in; a.base = W1; a.src = s;
    a.dacc = D; a.dacc_init = i == 0; a.cacc = sc.b[i] * dt;
    a.Wout = out; a.cout = sc.cout[i] * dt; a.cd = sc.cd[i];
    if (last) { a.wbase = w; a.wout = wo; a.wout_mirror = wo_mirror; }
    if (ns::launch_rhs_stage<CT, CT, CT>(c->g, cf, a, c->st) != cudaSuccess) return NS_ERR_CUDA;
    in = out;
  }
  return NS_OK;
}

// One CUDA event of the profiling pairs (kernel profiling on): a pair brackets the
// consecutive adjoint-stage launches of one step.
static void prof_mark(ns_ctx* c) {
  if (!c->prof_on) return;
  if (c->prof_used == c->events.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return;
    c->events.push_back(ev);
  }
  cudaEventRecord(c->events[c->prof_used++], c->st);
}

template <class CT, class TIN, class TA, class TST>
static cudaError_t adj_launch(ns_ctx* c, const Coef<CT>& cf, const ns::AdjArgs<TIN, TA, TST>& a) {
  if (c->prof_on) ++c->prof_launches;
  return ns::launch_adj_stage<CT, TIN, TA, TST>(c->g, cf, a, c->st);
}

// Recompute the stage states W2..W_ns from W1 = w^n (unless kept), then the transposed
// stages last to first with the stage products summed in the stage type and
// lam^n = lam^{n+1} + G formed in FP64.
template <class CT>
static int adjoint_step_t(ns_ctx* c, const Coef<CT>& cf, const CT* W1, const CT* lamf, const double* s,
                          const double* lam, const float* nu, double* lo, double* sbar,
                          const CT* const* kept = nullptr, CT* lo_mirror = nullptr, const double* nud = nullptr,
                          const ns_obj_src* obj = nullptr) {
  const Scheme& sc = scheme_of(c);
  const double dt = c->p.dt;
  const CT* Wst[3];
  CT* Aa = buf<CT>(c, AA);
  CT* Ab = buf<CT>(c, AB);
  CT* G = buf<CT>(c, GS);
  CT* S = buf<CT>(c, SB);
  if (kept) {
    // stage states kept by the replay of this step
    for (int i = 0; i < sc.ns - 1; ++i) Wst[i] = kept[i];
  } else {
    // G doubles as the increment sum of the recompute when the tableau needs it
    const int wb[3] = {W2, W3, W4};
    const CT* in = W1;
    for (int i = 0; i < sc.ns - 1; ++i) {
      CT* out = buf<CT>(c, wb[i]);
      ns::StageArgs<CT, CT> a{};
      a.W = in; a.base = W1; a.src = s; a.Wout = out; a.cout = sc.cout[i] * dt; a.cd = sc.cd[i];
      if (sc.needs_sum()) { a.dacc = G; a.dacc_init = i == 0; a.cacc = sc.b[i] * dt; }
      if (ns::launch_rhs_stage<CT, CT, CT>(c->g, cf, a, c->st) != cudaSuccess) return NS_ERR_CUDA;
      Wst[i] = out;
      in = out;
    }
  }
  const CT* Ain = lamf;
  prof_mark(c);
  for (int j = 0; j < sc.ns; ++j) {
    const bool last = j == sc.ns - 1;
    CT* Aout = last ? nullptr : (j % 2 == 0 ? Aa : Ab);
    ns::AdjArgs<CT, CT, CT> a{};
    a.W = last ? W1 : Wst[sc.ns - 2 - j];
    a.A = Ain; a.ca = j == 0 ? sc.ca0 * dt : 1.0; a.nu = nu; a.nud = nu ? nullptr : nud; a.lamf = lamf;
    for (int q = 0; q < 3; ++q) a.nus[q] = c->nu_split[q];
    a.Gin = j == 0 ? nullptr : G;
    a.Anext = Aout;
    if (!last) { a.cl = sc.cl[j] * dt; a.cg = sc.cg[j] * dt; a.cs = sc.cs[j] * dt; }
    if (!last) {
      a.Gout = G;
    } else {
      a.lam_in = lam;
      a.lam_out = lo;
      a.lam_out_mirror = lo_mirror;
      if (obj) {
        a.obj_aface = obj->aface;
        a.obj_ndsc = obj->ndsc;
        a.obj_iL = obj->iL;
        a.obj_iR = obj->iR;
      }
    }
    if (sbar) {
      a.SBin = j == 0 ? nullptr : S;
      if (!last) a.SBout = S; else a.sbar = sbar;
    }
    if (adj_launch(c, cf, a) != cudaSuccess) return NS_ERR_CUDA;
    Ain = Aout;
  }
  prof_mark(c);
  return NS_OK;
}

// ---------------------------------------------------------------------------------
// bounded boxes (ns_set_boundaries): the calls below run the periodic stage kernels on
// the box padded by its ghost layer (ns_bc.cu), filling the ghosts of every stage state
// they form, and crop the results
// ---------------------------------------------------------------------------------
template <class CT>
static CT* bW(ns_ctx* c, int i) {
  return (CT*)c->bstage[i];
}

template <class CT>
static const Coef<CT>& bcoef(const ns_ctx* c);
template <>
const Coef<float>& bcoef<float>(const ns_ctx* c) { return c->cf; }
template <>
const Coef<double>& bcoef<double>(const ns_ctx* c) { return c->cd; }

// W1 (padded, stage type) = w with its ghost layer; the source padded with zero ghosts
template <class CT>
static int bounded_prepare(ns_ctx* c, const double* w, const double* s, const double** sp) {
  if (ns::launch_bc_embed<CT, double>(c->g, c->bc, 5, 1.0, w, bW<CT>(c, 0), c->st) != cudaSuccess ||
      ns::launch_bc_ghosts<CT>(c->g, c->bc, bW<CT>(c, 0), c->st) != cudaSuccess)
    return NS_ERR_CUDA;
  *sp = nullptr;
  if (s) {
    if (ns::launch_bc_embed<double, double>(c->g, c->bc, 5, 1.0, s, c->bd[2], c->st) != cudaSuccess)
      return NS_ERR_CUDA;
    *sp = c->bd[2];
  }
  return NS_OK;
}

// stage i of the padded step: W_{i+1} with its ghosts (not last) or the padded FP64
// output (last, base = the padded state w)
template <class CT>
static int bounded_stage(ns_ctx* c, int i, bool final_out, const double* sp, bool with_sum) {
  const Scheme& sc = scheme_of(c);
  const double dt = c->p.dt;
  const bool last = final_out && i == sc.ns - 1;
  ns::StageArgs<CT, CT> a{};
  a.W = bW<CT>(c, i); a.base = bW<CT>(c, 0); a.src = sp;
  if (with_sum) { a.dacc = bW<CT>(c, 4); a.dacc_init = i == 0; a.cacc = sc.b[i] * dt; }
  if (!last) { a.Wout = bW<CT>(c, i + 1); a.cout = sc.cout[i] * dt; a.cd = sc.cd[i]; }
  else { a.wbase = c->bd[0]; a.wout = c->bd[1]; }
  if (ns::launch_rhs_stage<CT, CT, CT>(c->gp, bcoef<CT>(c), a, c->st) != cudaSuccess) return NS_ERR_CUDA;
  if (!last && ns::launch_bc_ghosts<CT>(c->g, c->bc, bW<CT>(c, i + 1), c->st) != cudaSuccess) return NS_ERR_CUDA;
  return NS_OK;
}

template <class CT>
static int bounded_primal_t(ns_ctx* c, const double* w, const double* s, double* wo) {
  const double* sp = nullptr;
  int r = bounded_prepare<CT>(c, w, s, &sp);
  if (r) return r;
  if (ns::launch_bc_embed<double, double>(c->g, c->bc, 5, 1.0, w, c->bd[0], c->st) != cudaSuccess)
    return NS_ERR_CUDA;
  const Scheme& sc = scheme_of(c);
  for (int i = 0; i < sc.ns; ++i)
    if ((r = bounded_stage<CT>(c, i, true, sp, true))) return r;
  return cuerr(ns::launch_bc_crop<double, double>(c->g, c->bc, 5, c->bd[1], wo, c->st));
}

template <class CT>
static int bounded_rhs_t(ns_ctx* c, const double* w, const double* s, double* R) {
  const double* sp = nullptr;
  int r = bounded_prepare<CT>(c, w, s, &sp);
  if (r) return r;
  ns::StageArgs<CT, CT> a{};
  a.W = bW<CT>(c, 0); a.src = sp; a.cacc = 1.0; a.wout = c->bd[1];
  if (ns::launch_rhs_stage<CT, CT, CT>(c->gp, bcoef<CT>(c), a, c->st) != cudaSuccess) return NS_ERR_CUDA;
  return cuerr(ns::launch_bc_crop<double, double>(c->g, c->bc, 5, c->bd[1], R, c->st));
}

// the transposed product on the padded box of seed sa*A at padded stage state W
// (into bd[3]), then the boundary epilogue e
template <class CT, class NU>
static int bounded_transposed_stage(ns_ctx* c, const CT* W, ns::BcEpilogue& e, const NU* nu) {
  if (ns::launch_bc_embed<CT, double>(c->g, c->bc, 5, e.sa, e.A, bW<CT>(c, 5), c->st) != cudaSuccess)
    return NS_ERR_CUDA;
  ns::AdjArgs<CT, CT, CT> a{};
  a.W = W; a.A = bW<CT>(c, 5); a.ca = 1.0; a.lam_out = c->bd[3];
  if (ns::launch_adj_stage<CT, CT, CT, CT>(c->gp, bcoef<CT>(c), a, c->st) != cudaSuccess) return NS_ERR_CUDA;
  for (int q = 0; q < 3; ++q) e.nus[q] = c->nu_split[q];
  e.i2[0] = 1.0 / (c->p.dx * c->p.dx);
  e.i2[1] = 1.0 / (c->p.dy * c->p.dy);
  e.i2[2] = 1.0 / (c->p.dz * c->p.dz);
  return cuerr(ns::launch_bc_adj_epilogue<CT, NU>(c->g, c->bc, e, c->bd[3], W, nu, c->st));
}

template <class CT>
static int bounded_transposed(ns_ctx* c, const CT* W, ns::BcEpilogue& e, const float* nu, const double* nud) {
  if (nud) return bounded_transposed_stage<CT, double>(c, W, e, nud);
  return bounded_transposed_stage<CT, float>(c, W, e, nu);
}

template <class CT>
static int bounded_transpose_t(ns_ctx* c, const double* w, const double* a_, const float* nu, double* out) {
  const double* sp = nullptr;
  int r = bounded_prepare<CT>(c, w, nullptr, &sp);
  if (r) return r;
  ns::BcEpilogue e{};
  e.A = a_; e.sa = 1.0; e.mode = 0; e.out = out;
  return bounded_transposed<CT>(c, bW<CT>(c, 0), e, nu, nullptr);
}

template <class CT>
static int bounded_adjoint_t(ns_ctx* c, const double* w, const double* s, const double* lam, const float* nu,
                             const double* nud, double* lo, double* sbar) {
  const Scheme& sc = scheme_of(c);
  const double dt = c->p.dt;
  const double* sp = nullptr;
  int r = bounded_prepare<CT>(c, w, s, &sp);
  if (r) return r;
  for (int i = 0; i < sc.ns - 1; ++i)
    if ((r = bounded_stage<CT>(c, i, false, sp, sc.needs_sum()))) return r;
  const double* Ain = lam;
  double sa = sc.ca0 * dt;
  for (int j = 0; j < sc.ns; ++j) {
    const bool last = j == sc.ns - 1;
    const CT* W = bW<CT>(c, last ? 0 : sc.ns - 1 - j);
    ns::BcEpilogue e{};
    e.A = Ain; e.sa = sa; e.mode = 1; e.first = j == 0; e.last = last;
    e.lam = lam; e.G = c->ba[2];
    if (!last) { e.cl = sc.cl[j] * dt; e.cg = sc.cg[j] * dt; e.cs = sc.cs[j] * dt; e.a_next = c->ba[j % 2]; }
    else e.out = lo;
    e.sbar = sbar;
    if ((r = bounded_transposed<CT>(c, W, e, nu, nud))) return r;
    Ain = e.a_next;
    sa = 1.0;
  }
  return NS_OK;
}

template <class CT>
static int bounded_sigma1_t(ns_ctx* c, const double* w, float* sigma1, double* sigma1d) {
  const double* sp = nullptr;
  int r = bounded_prepare<CT>(c, w, nullptr, &sp);
  if (r) return r;
  if (ns::launch_sigma1<CT>(c->gp, bcoef<CT>(c), bW<CT>(c, 0), sigma1 ? (float*)c->bsig : nullptr, nullptr,
                            c->scratch, c->ticket, c->st, nullptr,
                            sigma1d ? (double*)c->bsig : nullptr) != cudaSuccess)
    return NS_ERR_CUDA;
  if (sigma1d) return cuerr(ns::launch_bc_crop<double, double>(c->g, c->bc, 1, (double*)c->bsig, sigma1d, c->st));
  return cuerr(ns::launch_bc_crop<float, float>(c->g, c->bc, 1, (float*)c->bsig, sigma1, c->st));
}

static void free_bounded(ns_ctx* c) {
  for (void*& q : c->bstage) { if (q) cudaFree(q); q = nullptr; }
  for (double*& q : c->bd) { if (q) cudaFree(q); q = nullptr; }
  for (double*& q : c->ba) { if (q) cudaFree(q); q = nullptr; }
  if (c->bsig) cudaFree(c->bsig);
  c->bsig = nullptr;
}

extern "C" {

const char* ns_error_string(int code) {
  switch (code) {
    case NS_OK: return "ok";
    case NS_ERR_ARG: return "invalid argument";
    case NS_ERR_BUDGET: return "memory budget too small";
    case NS_ERR_NONFINITE: return "non-finite value detected";
    case NS_ERR_UNSTABLE: return "adjoint viscosity exceeds the explicit stability limit";
    case NS_ERR_CUDA: return "CUDA error";
    case NS_ERR_CORRUPT: return "a checkpoint snapshot changed between store and load";
    case NS_ERR_BOUNDS: return "a field index outside its field (bounds-checking build)";
    case NS_ERR_IO: return "the checkpoint snapshot file could not be created, written or read";
    default: return "unknown error";
  }
}

int ns_create(const ns_params* p, void* stream, ns_ctx** out) {
  if (!p || !out) return NS_ERR_ARG;
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->batch < 1) return NS_ERR_ARG;
  if (!(p->dx > 0) || !(p->dy > 0) || !(p->dz > 0) || !(p->gamma > 1.0) || !(p->mu >= 0) ||
      !(p->Pr > 0) || !(p->dt >= 0))
    return NS_ERR_ARG;
  if (p->precision != NS_FP64 && p->precision != NS_MIXED) return NS_ERR_ARG;
  if (p->scheme != NS_RK4 && p->scheme != NS_SSPRK3) return NS_ERR_ARG;
  if (p->flux != NS_FLUX_CENTRAL && p->flux != NS_FLUX_ROE) return NS_ERR_ARG;
  if (p->flux == NS_FLUX_ROE && !(p->roe_delta > 0.0 && p->roe_delta < 1e30)) return NS_ERR_ARG;
  if ((long long)p->nx * p->ny > (1LL << 31) || (long long)p->nx * p->ny * p->nz > (1LL << 40))
    return NS_ERR_ARG;
  if (p->plane_i <= -(1 << 30) || p->plane_i >= (1 << 30)) return NS_ERR_ARG;
  ns_ctx* c = new ns_ctx();
  c->p = *p;
  c->st = (cudaStream_t)stream;
  c->g.nx = p->nx;
  c->g.ny = p->ny;
  c->g.nz = p->nz;
  c->g.batch = p->batch;
  c->g.plane = (long long)p->nx * p->ny;
  c->g.cells = c->g.plane * p->nz;
  c->cd = make_coef<double>(*p);
  c->cf = make_coef<float>(*p);
  {
    Coef<double> d = c->cd;
    Coef<Dual>& x = c->cx;
    x.gamma = Dual(d.gamma);
    x.gm1 = Dual(d.gm1);
    x.mu = Dual(d.mu);
    x.alpha = Dual(d.alpha);
    x.roe_delta = Dual(d.roe_delta);
    x.roe = d.roe;
    for (int i = 0; i < 3; ++i) {
      x.idx[i] = Dual(d.idx[i]);
      x.i4dx[i] = Dual(d.i4dx[i]);
      x.hidx[i] = Dual(d.hidx[i]);
    }
  }
  c->field = (size_t)5 * c->g.cells * p->batch;
  const size_t esz = p->precision == NS_MIXED ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < ns_ctx::NSTAGE && e == cudaSuccess; ++i) e = cudaMalloc(&c->stage[i], c->field * esz);
  c->scratch_n = std::max(ns::diag_scratch_doubles(c->g, 256), ns::box_means_scratch_doubles(c->g));
  if (e == cudaSuccess) e = cudaMalloc(&c->scratch, c->scratch_n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&c->qbar, sizeof(double) * 5 * p->batch);
  if (e == cudaSuccess) e = cudaMalloc(&c->ticket, sizeof(unsigned) * p->batch);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ticket, 0, sizeof(unsigned) * p->batch, c->st);
  // the side stream of the sweep's objective sums: partials, (N/D, sc) and the per-face
  // factors of launch_objective_sum
  const size_t on = ns::objective_scratch_doubles(c->g) + (size_t)c->g.ny * c->g.nz * c->g.batch * 5;
  if (e == cudaSuccess) e = cudaMalloc(&c->oscratch, on * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->oticket, sizeof(unsigned) * p->batch);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->oticket, 0, sizeof(unsigned) * p->batch, c->st);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->ost, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ofork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ojoin, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    ns_destroy(c);
    return NS_ERR_CUDA;
  }
  c->ws_bytes = ns_ctx::NSTAGE * c->field * esz + c->scratch_n * sizeof(double) + sizeof(unsigned);
  c->g.dbg_err = c->err;   // the bounds checks of debug builds report here
  *out = c;
  return NS_OK;
}

void ns_destroy(ns_ctx* c) {
  if (!c) return;
  ns_sweep_release(c);
  if (c->rctx) ns_destroy(c->rctx);
  for (int i = 0; i < ns_ctx::NSTAGE; ++i)
    if (c->stage[i]) cudaFree(c->stage[i]);
  for (int i = 0; i < 6; ++i)
    if (c->tan[i]) cudaFree(c->tan[i]);
  if (c->scratch) cudaFree(c->scratch);
  if (c->own_err) {
    cudaFree(c->own_err);   // a replay context: err is its owner's
  } else if (c->err) {
    cudaFree(c->err);
  }
  if (c->qbar) cudaFree(c->qbar);
  if (c->ticket) cudaFree(c->ticket);
  if (c->oscratch) cudaFree(c->oscratch);
  if (c->oticket) cudaFree(c->oticket);
  if (c->ofork) cudaEventDestroy(c->ofork);
  if (c->ojoin) cudaEventDestroy(c->ojoin);
  if (c->ost) cudaStreamDestroy(c->ost);
  if (c->train_scratch) cudaFree(c->train_scratch);
  for (cudaEvent_t ev : c->events) cudaEventDestroy(ev);
  free_bounded(c);
  if (c->owns_stream) cudaStreamDestroy(c->st);
  delete c;
}

int ns_set_boundaries(ns_ctx* c, int bc, const double* far, const double* wall_e) {
  if (!c || bc < NS_BC_PERIODIC || bc > NS_BC_INOUT_WALLS) return NS_ERR_ARG;
  const int inout = bc == NS_BC_INOUT || bc == NS_BC_INOUT_WALLS;
  const int walls = bc == NS_BC_WALLS || bc == NS_BC_INOUT_WALLS;
  if ((inout && !far) || (walls && !wall_e)) return NS_ERR_ARG;
  if (inout && !(far[0] > 0 && far[4] > 0)) return NS_ERR_ARG;
  if (walls && !(wall_e[0] > 0 && wall_e[1] > 0)) return NS_ERR_ARG;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return NS_ERR_CUDA;
  free_bounded(c);
  c->bc = ns::BcDesc{};
  c->bc.gamma = c->p.gamma;
  if (!inout && !walls) return NS_OK;
  c->bc.inout = inout;
  c->bc.walls = walls;
  for (int k = 0; k < 5; ++k) c->bc.far[k] = inout ? far[k] : 0.0;
  for (int k = 0; k < 2; ++k) c->bc.wall_e[k] = walls ? wall_e[k] : 0.0;
  c->gp = c->g;
  c->gp.nx = c->g.nx + 2 * inout;
  c->gp.ny = c->g.ny + 2 * walls;
  c->gp.plane = (long long)c->gp.nx * c->gp.ny;
  c->gp.cells = c->gp.plane * c->gp.nz;
  const size_t np = (size_t)5 * c->gp.cells * c->p.batch, nc = (size_t)5 * c->g.cells * c->p.batch;
  const size_t esz = mixed(c) ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMalloc(&c->bstage[i], np * esz);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(&c->bd[i], np * sizeof(double));
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&c->ba[i], nc * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->bsig, (size_t)c->gp.cells * c->p.batch * sizeof(double));
  if (e != cudaSuccess) {
    free_bounded(c);
    c->bc = ns::BcDesc{};
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

int ns_set_stream(ns_ctx* c, void* stream) {
  if (!c) return NS_ERR_ARG;
  c->st = (cudaStream_t)stream;
  return NS_OK;
}

int ns_set_dt(ns_ctx* c, double dt) {
  if (!c || !(dt >= 0)) return NS_ERR_ARG;
  c->p.dt = dt;
  return NS_OK;
}

size_t ns_workspace_bytes(const ns_ctx* c) { return c ? c->ws_bytes : 0; }

int ns_rhs(ns_ctx* c, const double* w, const double* s, double* R) {
  if (!c || !w || !R || (const double*)R == w) return NS_ERR_ARG;
  if (c->bounded()) return mixed(c) ? bounded_rhs_t<float>(c, w, s, R) : bounded_rhs_t<double>(c, w, s, R);
  if (mixed(c)) {
    float* wf = buf<float>(c, WF);
    if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    ns::StageArgs<float, float> a{};
    a.W = wf; a.src = s; a.cacc = 1.0; a.wout = R;
    return cuerr(ns::launch_rhs_stage<float, float, float>(c->g, c->cf, a, c->st));
  }
  ns::StageArgs<double, double> a{};
  a.W = w; a.src = s; a.cacc = 1.0; a.wout = R;
  return cuerr(ns::launch_rhs_stage<double, double, double>(c->g, c->cd, a, c->st));
}

int ns_rhs_tangent(ns_ctx* c, const double* w, const double* wd, double* Rd) {
  if (!c || !w || !wd || !Rd || Rd == w || Rd == wd || c->bounded()) return NS_ERR_ARG;
  int r = ensure_tangent_buffers(c);
  if (r) return r;
  ns::StageArgs<double, double> a{};
  a.W = w; a.Wd = wd; a.cacc = 1.0; a.woutd = Rd;
  return cuerr(ns::launch_rhs_stage<Dual, double, double>(c->g, c->cx, a, c->st));
}

int ns_primal_step(ns_ctx* c, const double* w, const double* s, double* wo) {
  if (!c || !w || !wo || wo == w || wo == s) return NS_ERR_ARG;
  if (c->bounded()) return mixed(c) ? bounded_primal_t<float>(c, w, s, wo) : bounded_primal_t<double>(c, w, s, wo);
  if (mixed(c)) {
    float* wf = buf<float>(c, WF);
    if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    return primal_step_t<float>(c, c->cf, wf, w, s, wo);
  }
  return primal_step_t<double>(c, c->cd, w, w, s, wo);
}

int ns_tangent_step(ns_ctx* c, const double* w, const double* s, const double* wd, const double* sd,
                    double* wdo) {
  if (!c || !w || !wd || !wdo || wdo == wd || wdo == w || c->bounded()) return NS_ERR_ARG;
  int r = ensure_tangent_buffers(c);
  if (r) return r;
  const Scheme& sc = scheme_of(c);
  const double dt = c->p.dt;
  double *Wa = c->tan[0], *Wb = c->tan[1], *Wda = c->tan[2], *Wdb = c->tan[3], *D = c->tan[4],
         *Dd = c->tan[5];
  const double *in = w, *ind = wd;
  for (int i = 0; i < sc.ns; ++i) {
    const bool last = i == sc.ns - 1;
    double* out = last ? nullptr : (i % 2 == 0 ? Wa : Wb);
    double* outd = last ? nullptr : (i % 2 == 0 ? Wda : Wdb);
    ns::StageArgs<double, double> a{};
    a.W = in; a.Wd = ind;
    a.base = w; a.based = wd; a.src = s; a.srcd = sd;
    a.dacc = D; a.daccd = Dd; a.dacc_init = i == 0; a.cacc = sc.b[i] * dt;
    a.Wout = out; a.Woutd = outd; a.cout = sc.cout[i] * dt; a.cd = sc.cd[i];
    if (last) { a.wbased = wd; a.woutd = wdo; }
    if (ns::launch_rhs_stage<Dual, double, double>(c->g, c->cx, a, c->st) != cudaSuccess) return NS_ERR_CUDA;
    in = out;
    ind = outd;
  }
  return NS_OK;
}

int ns_adjoint_step(ns_ctx* c, const double* w, const double* s, const double* lam, const float* nu,
                    double* lo, double* sbar) {
  if (!c || !w || !lam || !lo || lo == lam || lo == w || (sbar && (sbar == lo || sbar == lam)))
    return NS_ERR_ARG;
  if (c->bounded())
    return mixed(c) ? bounded_adjoint_t<float>(c, w, s, lam, nu, nullptr, lo, sbar)
                    : bounded_adjoint_t<double>(c, w, s, lam, nu, nullptr, lo, sbar);
  if (mixed(c)) {
    float* wf = buf<float>(c, WF);
    float* lf = buf<float>(c, LF);
    if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    if (ns::launch_to_float(lam, lf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    return adjoint_step_t<float>(c, c->cf, wf, lf, s, lam, nu, lo, sbar);
  }
  return adjoint_step_t<double>(c, c->cd, w, lam, s, lam, nu, lo, sbar);
}

int ns_adjoint_step_f64(ns_ctx* c, const double* w, const double* s, const double* lam, const double* nu,
                        double* lo, double* sbar) {
  if (!c || mixed(c) || !w || !lam || !lo || lo == lam || lo == w || (sbar && (sbar == lo || sbar == lam)))
    return NS_ERR_ARG;
  if (c->bounded()) return bounded_adjoint_t<double>(c, w, s, lam, nullptr, nu, lo, sbar);
  return adjoint_step_t<double>(c, c->cd, w, lam, s, lam, nullptr, lo, sbar, nullptr, nullptr, nu);
}

int ns_rhs_transpose(ns_ctx* c, const double* w, const double* a_, const float* nu, double* out) {
  if (!c || !w || !a_ || !out || out == w || out == a_) return NS_ERR_ARG;
  if (c->bounded())
    return mixed(c) ? bounded_transpose_t<float>(c, w, a_, nu, out) : bounded_transpose_t<double>(c, w, a_, nu, out);
  if (mixed(c)) {
    float* wf = buf<float>(c, WF);
    float* af = buf<float>(c, LF);
    if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    if (ns::launch_to_float(a_, af, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    ns::AdjArgs<float, float, float> a{};
    a.W = wf; a.A = af; a.ca = 1.0; a.nu = nu; a.lam_out = out;
    for (int q = 0; q < 3; ++q) a.nus[q] = c->nu_split[q];
    return cuerr(ns::launch_adj_stage<float, float, float, float>(c->g, c->cf, a, c->st));
  }
  ns::AdjArgs<double, double, double> a{};
  a.W = w; a.A = a_; a.ca = 1.0; a.nu = nu; a.lam_out = out;
  for (int q = 0; q < 3; ++q) a.nus[q] = c->nu_split[q];
  return cuerr(ns::launch_adj_stage<double, double, double, double>(c->g, c->cd, a, c->st));
}

int ns_objective(ns_ctx* c, const double* w, double weight, double* J_acc, double* lam) {
  if (!c || !w || !J_acc || lam == w) return NS_ERR_ARG;
  const int i0 = c->p.plane_i;
  return cuerr(ns::launch_objective_fast(c->g, c->p.gamma, i0, c->p.pt_in, w, weight, J_acc, lam, c->err,
                                         c->scratch, c->ticket, c->st));
}

int ns_growth_sigma1(ns_ctx* c, const double* w, float* sigma1, double* stats) {
  if (!c || !w || !sigma1) return NS_ERR_ARG;
  if (c->bounded()) {
    if (stats) return NS_ERR_ARG;
    return mixed(c) ? bounded_sigma1_t<float>(c, w, sigma1, nullptr) : bounded_sigma1_t<double>(c, w, sigma1, nullptr);
  }
  if (mixed(c)) {
    float* wf = buf<float>(c, WF);
    if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    return cuerr(ns::launch_sigma1<float>(c->g, c->cf, wf, sigma1, stats, c->scratch, c->ticket, c->st));
  }
  return cuerr(ns::launch_sigma1<double>(c->g, c->cd, w, sigma1, stats, c->scratch, c->ticket, c->st));
}

int ns_growth_sigma1_f64(ns_ctx* c, const double* w, double* sigma1, double* stats) {
  if (!c || mixed(c) || !w || !sigma1) return NS_ERR_ARG;
  if (c->bounded()) return stats ? NS_ERR_ARG : bounded_sigma1_t<double>(c, w, nullptr, sigma1);
  return cuerr(ns::launch_sigma1<double>(c->g, c->cd, w, nullptr, stats, c->scratch, c->ticket, c->st, nullptr,
                                         sigma1));
}

static double nu_limit(const ns_ctx* c) {
  const double k = 4.0 * (1.0 / (c->p.dx * c->p.dx) + 1.0 / (c->p.dy * c->p.dy) +
                          (c->p.nz > 1 ? 1.0 / (c->p.dz * c->p.dz) : 0.0));
  const double f = std::max(c->nu_split[0], std::max(c->nu_split[1], c->nu_split[2]));
  return c->p.dt > 0 && f > 0 ? scheme_of(c).limit / (c->p.dt * k * f) : INFINITY;
}

int ns_add_adjoint_viscosity(ns_ctx* c, const float* sigma1, double lambda, double tau, float* nu) {
  if (!c || !sigma1 || !nu || !(lambda >= 0)) return NS_ERR_ARG;
  const double limit = nu_limit(c);
  return cuerr(ns::launch_nu_rule(c->g, sigma1, lambda, tau, limit, nu, c->err, c->st, c->nu_cap != 0));
}

int ns_add_adjoint_viscosity_f64(ns_ctx* c, const double* sigma1, double lambda, double tau, double* nu) {
  if (!c || !sigma1 || !nu || !(lambda >= 0)) return NS_ERR_ARG;
  return cuerr(ns::launch_nu_rule_f64(c->g, sigma1, lambda, tau, nu_limit(c), nu, c->err, c->st, c->nu_cap != 0));
}

int ns_apply_adjoint_viscosity(ns_ctx* c, const float* nu, const double* a, double* out) {
  if (!c || !nu || !a || !out || out == a || c->bounded()) return NS_ERR_ARG;
  const double i2[3] = {1.0 / (c->p.dx * c->p.dx), 1.0 / (c->p.dy * c->p.dy), 1.0 / (c->p.dz * c->p.dz)};
  return cuerr(ns::launch_visc_apply(c->g, i2, c->nu_split, nu, a, out, c->st));
}

int ns_adjoint_energy(ns_ctx* c, const double* w, const double* lam, double* E) {
  if (!c || !w || !lam || !E) return NS_ERR_ARG;
  const double dV = c->p.dx * c->p.dy * c->p.dz;
  return cuerr(ns::launch_energy(c->g, c->p.gamma, dV, w, lam, E, c->scratch, c->err, mixed(c), c->ticket,
                                 c->st));
}

int ns_dot(ns_ctx* c, const double* a, const double* phi, int nphi, size_t n, double* out) {
  if (!c || !a || !phi || !out || nphi < 1 || nphi > 256 || n == 0) return NS_ERR_ARG;
  return cuerr(ns::launch_dot(a, phi, nphi, n, out, c->scratch, c->st));
}

int ns_combine(ns_ctx* c, const double* theta, const double* phi, int nphi, size_t n, double* s) {
  if (!c || !theta || !phi || !s || nphi < 1 || n == 0) return NS_ERR_ARG;
  return cuerr(ns::launch_combine(theta, phi, nphi, n, s, c->st));
}

int ns_scale_boxes(ns_ctx* c, const double* seed, double* field) {
  if (!c || !seed || !field) return NS_ERR_ARG;
  return cuerr(ns::launch_scale_boxes(c->g, seed, field, c->st));
}

int ns_dot_boxes(ns_ctx* c, const double* field, int comp, const double* phi, int nphi, double* out) {
  if (!c || !field || !phi || !out || comp < 0 || comp > 4 || nphi < 1 || nphi > 256) return NS_ERR_ARG;
  return cuerr(ns::launch_dot_boxes(c->g, field, comp, phi, nphi, out, c->scratch, c->st));
}

size_t ns_mlp_net_bytes(void) { return ns::MLP_BYTES; }

int ns_mlp_set_params(ns_ctx* c, void* net, const float* params) {
  if (!c || !net || !params) return NS_ERR_ARG;
  return cuerr(ns::launch_mlp_set(net, params, c->st));
}

int ns_mlp_get_params(ns_ctx* c, const void* net, float* params) {
  if (!c || !net || !params) return NS_ERR_ARG;
  return cuerr(cudaMemcpyAsync(params, (const char*)net + ns::MLP_OFF_MASTER, sizeof(float) * ns::NPAR,
                               cudaMemcpyDeviceToDevice, c->st));
}

int ns_mlp_get_moment(ns_ctx* c, const void* net, int which, float* out) {
  if (!c || !net || !out || (which != 1 && which != 2)) return NS_ERR_ARG;
  const size_t off = which == 1 ? ns::MLP_OFF_M : ns::MLP_OFF_V;
  return cuerr(cudaMemcpyAsync(out, (const char*)net + off, sizeof(float) * ns::NPAR, cudaMemcpyDeviceToDevice,
                               c->st));
}

int ns_mlp_features(ns_ctx* c, const double* w, float* feat) {
  if (!c || !w || !feat || c->bounded()) return NS_ERR_ARG;
  if (ns::launch_box_means(c->g, c->p.gamma, w, c->qbar, c->scratch, c->st) != cudaSuccess) return NS_ERR_CUDA;
  return cuerr(ns::launch_features(c->g, c->cf, w, c->qbar, feat, c->st));
}

int ns_mlp_infer(ns_ctx* c, const void* net, const float* feat, const float* sigma1, double kappa, float* nu) {
  if (!c || !net || !feat || !sigma1 || !nu || !(kappa >= 0)) return NS_ERR_ARG;
  const double scale = kappa * c->p.dx * c->p.dx;
  return cuerr(ns::launch_mlp_infer(c->g.cells * c->g.batch, const_cast<void*>(net), feat, sigma1, scale,
                                    nu_limit(c), nu, c->err, c->st, c->nu_cap != 0));
}

int ns_mlp_train_step(ns_ctx* c, void* net, const float* feat, const float* target, const int* idx, int n,
                      int step, double lr, float* loss) {
  if (!c || !net || !feat || !target || !idx || n < 1 || step < 1 || !(lr > 0)) return NS_ERR_ARG;
  const size_t need = ns::mlp_train_scratch_floats(n);
  if (need > c->train_scratch_n) {
    if (c->train_scratch) cudaFree(c->train_scratch);
    c->train_scratch = nullptr;
    c->train_scratch_n = 0;
    if (cudaMalloc(&c->train_scratch, need * sizeof(float)) != cudaSuccess) return NS_ERR_CUDA;
    c->train_scratch_n = need;
  }
  return cuerr(ns::launch_mlp_train_step(net, feat, target, idx, n, step, lr, c->train_scratch, loss, c->st));
}

int ns_adjoint_label(ns_ctx* c, const double* w, const double* lam, float* acc) {
  if (!c || !w || !lam || !acc || c->bounded()) return NS_ERR_ARG;
  if (mixed(c)) {
    float* wf = buf<float>(c, WF);
    if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
    return cuerr(ns::launch_label<float>(c->g, c->cf, wf, lam, acc, c->st));
  }
  return cuerr(ns::launch_label<double>(c->g, c->cd, w, lam, acc, c->st));
}

int ns_label_target(ns_ctx* c, const float* acc, const float* sigma1, double t_max, float* target) {
  if (!c || !acc || !sigma1 || !target || !(t_max > 0)) return NS_ERR_ARG;
  return cuerr(ns::launch_label_target(c->g.cells * c->g.batch, acc, sigma1, c->p.dx * c->p.dx, t_max, target,
                                       c->st));
}

int ns_to_float(ns_ctx* c, const double* in, float* out, size_t n) {
  if (!c || !in || !out || n == 0) return NS_ERR_ARG;
  return cuerr(ns::launch_to_float(in, out, n, c->st));
}

int ns_max_wave_speed(ns_ctx* c, const double* w, double* out) {
  if (!c || !w || !out) return NS_ERR_ARG;
  return cuerr(ns::launch_max_wave(c->g, c->p.gamma, w, out, c->scratch, c->st));
}

int ns_set_viscosity_cap(ns_ctx* c, int cap) {
  if (!c) return NS_ERR_ARG;
  c->nu_cap = cap != 0;
  return NS_OK;
}

int ns_set_viscosity_split(ns_ctx* c, const double* split) {
  if (!c || !split) return NS_ERR_ARG;
  for (int q = 0; q < 3; ++q)
    if (!(split[q] >= 0.0) || !std::isfinite(split[q])) return NS_ERR_ARG;
  for (int q = 0; q < 3; ++q) c->nu_split[q] = split[q];
  return NS_OK;
}

unsigned long long ns_launch_count(void) { return ns::g_launches.load(std::memory_order_relaxed); }

int ns_last_error(ns_ctx* c) {
  if (!c) return NS_ERR_ARG;
  unsigned h = 0;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaMemcpy(&h, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaMemset(c->err, 0, sizeof(unsigned)) != cudaSuccess) return NS_ERR_CUDA;
  if (h & ns::ERRBIT_BOUNDS) return NS_ERR_BOUNDS;
  if (h & ns::ERRBIT_CORRUPT) return NS_ERR_CORRUPT;
  if (h & ns::ERRBIT_NONFINITE) return NS_ERR_NONFINITE;
  if (h & ns::ERRBIT_UNSTABLE) return NS_ERR_UNSTABLE;
  return NS_OK;
}

}  // extern "C"

extern "C" int ns_profile_enable(ns_ctx* c, int on) {
  if (!c) return NS_ERR_ARG;
  if (on && !c->prof_on) {
    c->prof_used = 0;
    c->prof_launches = 0;
  }
  c->prof_on = on != 0;
  return NS_OK;
}

extern "C" int ns_profile_read(ns_ctx* c, double* ms, long long* launches) {
  if (!c || !ms || !launches) return NS_ERR_ARG;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return NS_ERR_CUDA;
  double tot = 0.0;
  for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, c->events[i], c->events[i + 1]) != cudaSuccess) return NS_ERR_CUDA;
    tot += t;
  }
  *ms = tot;
  *launches = c->prof_launches;
  c->prof_used = 0;
  c->prof_launches = 0;
  return NS_OK;
}

// ---------------------------------------------------------------------------------
// internal step variants used by the sweep executor (not part of the C ABI): optional
// float mirrors of the input/output states and kept stage states (stage-type buffers)
// ---------------------------------------------------------------------------------
int ns_i_primal(ns_ctx* c, const double* w, const void* w_mirror, const double* s, double* wo, void* wo_mirror,
                void* const* keep3) {
  if (mixed(c)) {
    const float* W1 = (const float*)w_mirror;
    if (!W1) {
      float* wf = buf<float>(c, WF);
      if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
      W1 = wf;
    }
    return primal_step_t<float>(c, c->cf, W1, w, s, wo, (float*)wo_mirror, (float* const*)keep3);
  }
  return primal_step_t<double>(c, c->cd, w, w, s, wo, nullptr, (double* const*)keep3);
}

int ns_i_objective_sum_forked(ns_ctx* c, const double* w, double weight, double* J_acc, ns_obj_src* obj) {
  const int nx = c->g.nx, i0 = c->p.plane_i;
  obj->iL = ((i0 - 1) % nx + nx) % nx;
  obj->iR = (i0 % nx + nx) % nx;
  if (cudaEventRecord(c->ofork, c->st) != cudaSuccess || cudaStreamWaitEvent(c->ost, c->ofork, 0) != cudaSuccess)
    return NS_ERR_CUDA;
  if (ns::launch_objective_sum(c->g, c->p.gamma, i0, c->p.pt_in, w, weight, J_acc, c->err, c->oscratch, c->oticket,
                               c->ost, &obj->aface, &obj->ndsc) != cudaSuccess)
    return NS_ERR_CUDA;
  return cudaEventRecord(c->ojoin, c->ost) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

int ns_i_objective_join(ns_ctx* c) {
  return cudaStreamWaitEvent(c->st, c->ojoin, 0) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

int ns_i_adjoint(ns_ctx* c, const double* w, const void* w_mirror, const void* const* kept3, const double* s,
                 const double* lam, const void* lam_mirror, const float* nu, double* lo, void* lo_mirror,
                 double* sbar, const double* nud, const ns_obj_src* obj) {
  if (mixed(c)) {
    const float* W1 = (const float*)w_mirror;
    if (!W1) {
      float* wf = buf<float>(c, WF);
      if (ns::launch_to_float(w, wf, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
      W1 = wf;
    }
    const float* lf = (const float*)lam_mirror;
    if (!lf) {
      float* t = buf<float>(c, LF);
      if (ns::launch_to_float(lam, t, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
      lf = t;
    }
    return adjoint_step_t<float>(c, c->cf, W1, lf, s, lam, nu, lo, sbar, (const float* const*)kept3,
                                 (float*)lo_mirror, nullptr, obj);
  }
  return adjoint_step_t<double>(c, c->cd, w, lam, s, lam, nu, lo, sbar, (const double* const*)kept3, nullptr,
                                nud, obj);
}

int ns_i_energy(ns_ctx* c, const double* w, const void* w_mirror, const double* lam, const void* lam_mirror,
                double* E) {
  if (mixed(c) && w_mirror && lam_mirror) {
    const double dV = c->p.dx * c->p.dy * c->p.dz;
    return cuerr(ns::launch_energy_mirrors(c->g, c->p.gamma, dV, (const float*)w_mirror, (const float*)lam_mirror,
                                           E, c->scratch, c->err, c->ticket, c->st));
  }
  return ns_adjoint_energy(c, w, lam, E);
}


int ns_i_sigma1_f64(ns_ctx* c, const double* w, double* sigma1, double* stats, double lambda, double tau,
                    double* nu) {
  ns::NuRule rule{0.f, 0.f, 0.f, nullptr, c->err, lambda, tau, nu_limit(c), nu, c->nu_cap};
  return cuerr(ns::launch_sigma1<double>(c->g, c->cd, w, nullptr, stats, c->scratch, c->ticket, c->st,
                                         nu ? &rule : nullptr, sigma1));
}

int ns_i_sigma1(ns_ctx* c, const double* w, const void* w_mirror, float* sigma1, double* stats, double lambda,
                double tau, float* nu) {
  ns::NuRule rule{(float)lambda, (float)tau, (float)nu_limit(c), nu, c->err, 0.0, 0.0, 0.0, nullptr, c->nu_cap};
  const ns::NuRule* rp = nu ? &rule : nullptr;
  if (mixed(c)) {
    const float* wf = (const float*)w_mirror;
    if (!wf) {
      float* t = buf<float>(c, WF);
      if (ns::launch_to_float(w, t, c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
      wf = t;
    }
    return cuerr(ns::launch_sigma1<float>(c->g, c->cf, wf, sigma1, stats, c->scratch, c->ticket, c->st, rp));
  }
  return cuerr(ns::launch_sigma1<double>(c->g, c->cd, w, sigma1, stats, c->scratch, c->ticket, c->st, rp));
}

int ns_i_mlp_features(ns_ctx* c, const double* w, const void* w_mirror, float* feat) {
  if (!mixed(c) || !w_mirror) return ns_mlp_features(c, w, feat);
  const float* wf = (const float*)w_mirror;
  if (ns::launch_box_means(c->g, c->p.gamma, wf, c->qbar, c->scratch, c->st) != cudaSuccess) return NS_ERR_CUDA;
  return cuerr(ns::launch_features(c->g, c->cf, wf, c->qbar, feat, c->st));
}

size_t ns_i_stage_bytes(const ns_ctx* c) { return c->field * (mixed(c) ? sizeof(float) : sizeof(double)); }

// ---------------------------------------------------------------------------------
// x-slab decomposition (section "Numerical methods": the solver's domain is split over
// MPI ranks).  Every slab is a box of its own, padded with one ghost column on each x
// side: columns 0 and nx-1 of a slab hold the neighbouring slabs' boundary columns, so
// the periodic stencils of the stage kernels, run on the padded slab, give the exact
// result in its interior columns (the residual and its transpose reach one cell in x).
// Every stage of a step runs on all slabs, then the stage's output field is exchanged
// (one strided copy per halo); the stage products and sums stay per cell.  The slabs
// are periodic in x as a whole: slab 0's left neighbour is the last slab.
// ---------------------------------------------------------------------------------
struct ns_slab_group {
  std::vector<ns_ctx*> c;
  std::vector<cudaEvent_t> done, copied;
  ns_halo_exchange_fn fn = nullptr;   // host exchange (one slab per process), or null
  void* user = nullptr;
};

static int slab_exchange(ns_slab_group* G, void* const* f, int eb, int ncomp) {
  const int n = (int)G->c.size();
  if (G->fn) {
    for (int k = 0; k < n; ++k)
      if (G->fn(G->user, f[k], eb, ncomp) != 0) return NS_ERR_CUDA;
    return NS_OK;
  }
  // producers done on every stream before any copy reads a neighbour's columns
  for (int k = 0; k < n; ++k)
    if (cudaEventRecord(G->done[k], G->c[k]->st) != cudaSuccess) return NS_ERR_CUDA;
  for (int k = 0; k < n; ++k) {
    ns_ctx* c = G->c[k];
    const int L = (k + n - 1) % n, R = (k + 1) % n;
    if (cudaStreamWaitEvent(c->st, G->done[L], 0) != cudaSuccess ||
        cudaStreamWaitEvent(c->st, G->done[R], 0) != cudaSuccess)
      return NS_ERR_CUDA;
    const size_t rows = (size_t)c->g.batch * ncomp * c->g.nz * c->g.ny;
    const int nxk = c->g.nx, nxl = G->c[L]->g.nx, nxr = G->c[R]->g.nx;
    char* dst = (char*)f[k];
    // left ghost <- the left slab's last interior column; right ghost <- the right
    // slab's first interior column
    if (cudaMemcpy2DAsync(dst, (size_t)nxk * eb, (const char*)f[L] + (size_t)(nxl - 2) * eb, (size_t)nxl * eb, eb,
                          rows, cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      return NS_ERR_CUDA;
    if (cudaMemcpy2DAsync(dst + (size_t)(nxk - 1) * eb, (size_t)nxk * eb, (const char*)f[R] + (size_t)eb,
                          (size_t)nxr * eb, eb, rows, cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      return NS_ERR_CUDA;
  }
  // a neighbour's next kernel may overwrite the columns just read: it waits for the copies
  for (int k = 0; k < n; ++k)
    if (cudaEventRecord(G->copied[k], G->c[k]->st) != cudaSuccess) return NS_ERR_CUDA;
  for (int k = 0; k < n; ++k) {
    const int L = (k + n - 1) % n, R = (k + 1) % n;
    if (cudaStreamWaitEvent(G->c[k]->st, G->copied[L], 0) != cudaSuccess ||
        cudaStreamWaitEvent(G->c[k]->st, G->copied[R], 0) != cudaSuccess)
      return NS_ERR_CUDA;
  }
  return NS_OK;
}

template <class CT>
static const Coef<CT>& coef_of(const ns_ctx* c);
template <>
const Coef<float>& coef_of<float>(const ns_ctx* c) { return c->cf; }
template <>
const Coef<double>& coef_of<double>(const ns_ctx* c) { return c->cd; }

// the stages of primal_step_t on every slab, with the stage outputs exchanged
template <class CT>
static int slab_primal_t(ns_slab_group* G, const CT* const* W1, const double* const* w, const double* const* s,
                         double* const* wo) {
  const int n = (int)G->c.size();
  const Scheme& sc = scheme_of(G->c[0]);
  const double dt = G->c[0]->p.dt;
  std::vector<const CT*> in(W1, W1 + n);
  std::vector<void*> out(n);
  for (int i = 0; i < sc.ns; ++i) {
    const bool last = i == sc.ns - 1;
    for (int k = 0; k < n; ++k) {
      ns_ctx* c = G->c[k];
      CT* o = last ? nullptr : buf<CT>(c, i % 2 == 0 ? W2 : W3);
      ns::StageArgs<CT, CT> a{};
      a.W = in[k]; a.base = W1[k]; a.src = s ? s[k] : nullptr;
      a.dacc = buf<CT>(c, GS); a.dacc_init = i == 0; a.cacc = sc.b[i] * dt;
      a.Wout = o; a.cout = sc.cout[i] * dt; a.cd = sc.cd[i];
      if (last) { a.wbase = w[k]; a.wout = wo[k]; }
      if (ns::launch_rhs_stage<CT, CT, CT>(c->g, coef_of<CT>(c), a, c->st) != cudaSuccess) return NS_ERR_CUDA;
      out[k] = last ? (void*)wo[k] : (void*)o;
    }
    int r = slab_exchange(G, out.data(), last ? (int)sizeof(double) : (int)sizeof(CT), 5);
    if (r) return r;
    for (int k = 0; k < n; ++k) in[k] = (const CT*)out[k];
  }
  return NS_OK;
}

// the stages of adjoint_step_t (recompute, then the transposed stages) on every slab,
// with the recomputed stage states, the stage seeds and lam^n exchanged
template <class CT>
static int slab_adjoint_t(ns_slab_group* G, const CT* const* W1, const CT* const* lamf, const double* const* s,
                          const double* const* lam, const float* const* nu, double* const* lo) {
  const int n = (int)G->c.size();
  const Scheme& sc = scheme_of(G->c[0]);
  const double dt = G->c[0]->p.dt;
  std::vector<std::vector<const CT*>> Wst(n, std::vector<const CT*>(3, nullptr));
  std::vector<void*> out(n);
  const int wb[3] = {W2, W3, W4};
  for (int i = 0; i < sc.ns - 1; ++i) {
    for (int k = 0; k < n; ++k) {
      ns_ctx* c = G->c[k];
      CT* o = buf<CT>(c, wb[i]);
      ns::StageArgs<CT, CT> a{};
      a.W = i == 0 ? W1[k] : Wst[k][i - 1]; a.base = W1[k]; a.src = s ? s[k] : nullptr;
      a.Wout = o; a.cout = sc.cout[i] * dt; a.cd = sc.cd[i];
      if (sc.needs_sum()) { a.dacc = buf<CT>(c, GS); a.dacc_init = i == 0; a.cacc = sc.b[i] * dt; }
      if (ns::launch_rhs_stage<CT, CT, CT>(c->g, coef_of<CT>(c), a, c->st) != cudaSuccess) return NS_ERR_CUDA;
      Wst[k][i] = o;
      out[k] = o;
    }
    int r = slab_exchange(G, out.data(), (int)sizeof(CT), 5);
    if (r) return r;
  }
  std::vector<const CT*> Ain(lamf, lamf + n);
  for (int j = 0; j < sc.ns; ++j) {
    const bool last = j == sc.ns - 1;
    for (int k = 0; k < n; ++k) {
      ns_ctx* c = G->c[k];
      CT* Aout = last ? nullptr : buf<CT>(c, j % 2 == 0 ? AA : AB);
      ns::AdjArgs<CT, CT, CT> a{};
      a.W = last ? W1[k] : Wst[k][sc.ns - 2 - j];
      a.A = Ain[k]; a.ca = j == 0 ? sc.ca0 * dt : 1.0; a.nu = nu ? nu[k] : nullptr; a.lamf = lamf[k];
      for (int q = 0; q < 3; ++q) a.nus[q] = c->nu_split[q];
      a.Gin = j == 0 ? nullptr : buf<CT>(c, GS);
      a.Anext = Aout;
      if (!last) {
        a.cl = sc.cl[j] * dt; a.cg = sc.cg[j] * dt; a.cs = sc.cs[j] * dt;
        a.Gout = buf<CT>(c, GS);
      } else {
        a.lam_in = lam[k];
        a.lam_out = lo[k];
      }
      if (ns::launch_adj_stage<CT, CT, CT, CT>(c->g, coef_of<CT>(c), a, c->st) != cudaSuccess) return NS_ERR_CUDA;
      out[k] = last ? (void*)lo[k] : (void*)Aout;
    }
    int r = slab_exchange(G, out.data(), last ? (int)sizeof(double) : (int)sizeof(CT), 5);
    if (r) return r;
    for (int k = 0; k < n; ++k) Ain[k] = (const CT*)out[k];
  }
  return NS_OK;
}

extern "C" {

int ns_slab_group_create(ns_ctx* const* slabs, int n, ns_slab_group** out) {
  if (!slabs || !out || n < 1) return NS_ERR_ARG;
  *out = nullptr;
  const ns_params& p0 = slabs[0] ? slabs[0]->p : ns_params{};
  for (int k = 0; k < n; ++k) {
    const ns_ctx* c = slabs[k];
    if (!c || c->p.nx < 3 || c->bounded()) return NS_ERR_ARG;
    const ns_params& p = c->p;
    if (p.ny != p0.ny || p.nz != p0.nz || p.batch != p0.batch || p.precision != p0.precision ||
        p.scheme != p0.scheme || p.flux != p0.flux || p.dt != p0.dt || p.dx != p0.dx || p.dy != p0.dy ||
        p.dz != p0.dz || p.gamma != p0.gamma || p.mu != p0.mu || p.Pr != p0.Pr || p.roe_delta != p0.roe_delta)
      return NS_ERR_ARG;
  }
  ns_slab_group* G = new ns_slab_group();
  G->c.assign(slabs, slabs + n);
  G->done.assign(n, nullptr);
  G->copied.assign(n, nullptr);
  for (int k = 0; k < n; ++k) {
    if (cudaEventCreateWithFlags(&G->done[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->copied[k], cudaEventDisableTiming) != cudaSuccess) {
      ns_slab_group_destroy(G);
      return NS_ERR_CUDA;
    }
  }
  *out = G;
  return NS_OK;
}

void ns_slab_group_destroy(ns_slab_group* G) {
  if (!G) return;
  for (cudaEvent_t e : G->done)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : G->copied)
    if (e) cudaEventDestroy(e);
  delete G;
}

int ns_slab_set_exchange(ns_slab_group* G, ns_halo_exchange_fn fn, void* user) {
  if (!G || (fn && G->c.size() != 1)) return NS_ERR_ARG;
  G->fn = fn;
  G->user = user;
  return NS_OK;
}

int ns_slab_exchange(ns_slab_group* G, void* const* fields, int elem_bytes, int ncomp) {
  if (!G || !fields || (elem_bytes != 4 && elem_bytes != 8) || ncomp < 1) return NS_ERR_ARG;
  for (size_t k = 0; k < G->c.size(); ++k)
    if (!fields[k]) return NS_ERR_ARG;
  return slab_exchange(G, fields, elem_bytes, ncomp);
}

int ns_slab_primal_step(ns_slab_group* G, const double* const* w, const double* const* s, double* const* wo) {
  if (!G || !w || !wo) return NS_ERR_ARG;
  const int n = (int)G->c.size();
  for (int k = 0; k < n; ++k)
    if (!w[k] || !wo[k] || wo[k] == w[k] || (s && wo[k] == s[k])) return NS_ERR_ARG;
  if (mixed(G->c[0])) {
    std::vector<const float*> W1(n);
    for (int k = 0; k < n; ++k) {
      float* wf = buf<float>(G->c[k], WF);
      if (ns::launch_to_float(w[k], wf, G->c[k]->field, G->c[k]->st) != cudaSuccess) return NS_ERR_CUDA;
      W1[k] = wf;
    }
    return slab_primal_t<float>(G, W1.data(), w, s, wo);
  }
  return slab_primal_t<double>(G, w, w, s, wo);
}

int ns_slab_adjoint_step(ns_slab_group* G, const double* const* w, const double* const* s,
                         const double* const* lam, const float* const* nu, double* const* lo) {
  if (!G || !w || !lam || !lo) return NS_ERR_ARG;
  const int n = (int)G->c.size();
  for (int k = 0; k < n; ++k)
    if (!w[k] || !lam[k] || !lo[k] || lo[k] == lam[k] || lo[k] == w[k] || (nu && !nu[k])) return NS_ERR_ARG;
  if (mixed(G->c[0])) {
    std::vector<const float*> W1(n), lf(n);
    for (int k = 0; k < n; ++k) {
      ns_ctx* c = G->c[k];
      float* wf = buf<float>(c, WF);
      float* lm = buf<float>(c, LF);
      if (ns::launch_to_float(w[k], wf, c->field, c->st) != cudaSuccess ||
          ns::launch_to_float(lam[k], lm, c->field, c->st) != cudaSuccess)
        return NS_ERR_CUDA;
      W1[k] = wf;
      lf[k] = lm;
    }
    return slab_adjoint_t<float>(G, W1.data(), lf.data(), s, lam, nu, lo);
  }
  return slab_adjoint_t<double>(G, w, lam, s, lam, nu, lo);
}

// The checkpointed sweep on a slab group: the plan of ns_plan, each action on every slab
// (its states kept per slab), the objective and its source on slab `own`, the sigma_1
// rule's viscosity per slab with its ghost columns exchanged, lambda's ghost columns
// exchanged after every source.  Workspace of slab k: nbuf states, one adjoint field and,
// with the rule, sigma_1 and nu (float), each 256-byte aligned.
static size_t slab_state_bytes(const ns_ctx* c) { return (c->field * sizeof(double) + 255) & ~(size_t)255; }
static size_t slab_scalar_bytes(const ns_ctx* c) {
  return ((size_t)c->g.cells * c->g.batch * sizeof(float) + 255) & ~(size_t)255;
}

int ns_slab_run_bytes(ns_slab_group* G, const ns_run_opts* o, size_t* bytes) {
  if (!G || !o || !bytes) return NS_ERR_ARG;
  int nact = 0, slots = 0;
  long long adv = 0;
  int r = ns_plan(o->nsteps, o->schedule, o->param, nullptr, 0, &nact, &slots, &adv);
  if (r) return r;
  for (size_t k = 0; k < G->c.size(); ++k) {
    const ns_ctx* c = G->c[k];
    bytes[k] = (size_t)(slots + 3) * slab_state_bytes(c) + (o->lambda > 0.0 ? 2 * slab_scalar_bytes(c) : 0);
  }
  return NS_OK;
}

int ns_slab_adjoint_run(ns_slab_group* G, int own, const double* const* w0, const double* const* s,
                        const ns_run_opts* o, void* const* work, const size_t* work_bytes, double* Jbar,
                        double* const* lam0) {
  if (!G || !w0 || !o || !work || !work_bytes || !Jbar || !lam0) return NS_ERR_ARG;
  const int n = (int)G->c.size();
  if (own < 0 || own >= n) return NS_ERR_ARG;
  if (o->schedule != NS_CKPT_ALL && o->schedule != NS_CKPT_STRIDE && o->schedule != NS_CKPT_REVOLVE)
    return NS_ERR_ARG;
  if (o->mlp || o->record_energy || o->record_sigma || o->verify || !(o->lambda >= 0.0)) return NS_ERR_ARG;
  for (int k = 0; k < n; ++k)
    if (!w0[k] || !work[k] || !lam0[k] || lam0[k] == w0[k] || ((uintptr_t)work[k] & 255) != 0) return NS_ERR_ARG;
  int nact = 0, slots = 0;
  long long adv = 0;
  int r = ns_plan(o->nsteps, o->schedule, o->param, nullptr, 0, &nact, &slots, &adv);
  if (r) return r;
  std::vector<ns_action> acts(nact);
  if ((r = ns_plan(o->nsteps, o->schedule, o->param, acts.data(), nact, &nact, &slots, &adv))) return r;
  std::vector<size_t> need(n);
  if ((r = ns_slab_run_bytes(G, o, need.data()))) return r;
  for (int k = 0; k < n; ++k)
    if (work_bytes[k] < need[k]) return NS_ERR_BUDGET;
  // per slab: nbuf state buffers, the second adjoint field, sigma_1 and nu
  const int nbuf = slots + 2;
  std::vector<std::vector<double*>> buf(n, std::vector<double*>(nbuf));
  std::vector<double*> lamB(n);
  std::vector<float*> sig(n, nullptr), nu(n, nullptr);
  for (int k = 0; k < n; ++k) {
    char* q = (char*)work[k];
    const size_t st = slab_state_bytes(G->c[k]);
    for (int i = 0; i < nbuf; ++i) buf[k][i] = (double*)(q + (size_t)i * st);
    lamB[k] = (double*)(q + (size_t)nbuf * st);
    if (o->lambda > 0.0) {
      sig[k] = (float*)(q + (size_t)(nbuf + 1) * st);
      nu[k] = (float*)((char*)sig[k] + slab_scalar_bytes(G->c[k]));
    }
  }
  std::vector<int> slot_buf(std::max(slots, 1), -1);
  std::vector<char> owned(nbuf, 0);
  int cur = -1;   // -1: the caller's w0
  auto states = [&](int i) {
    std::vector<const double*> v(n);
    for (int k = 0; k < n; ++k) v[k] = i < 0 ? w0[k] : buf[k][i];
    return v;
  };
  auto pick_free = [&]() -> int {
    for (int i = 0; i < nbuf; ++i)
      if (!owned[i] && i != cur) return i;
    return -1;
  };
  // the adjoint fields alternate between lam0 and the workspace field, ending in lam0
  const int N = o->nsteps;
  std::vector<double*> lc(n), ln(n);
  for (int k = 0; k < n; ++k) {
    lc[k] = N % 2 == 0 ? lam0[k] : lamB[k];
    ln[k] = N % 2 == 0 ? lamB[k] : lam0[k];
  }
  ns_ctx* co = G->c[own];
  if (cudaMemsetAsync(Jbar, 0, (size_t)co->g.batch * sizeof(double), co->st) != cudaSuccess) return NS_ERR_CUDA;
  const double wN = 1.0 / N;
  for (const ns_action& A : acts) {
    switch (A.op) {
      case NS_OP_ADVANCE:
        for (int m = A.a; m < A.b; ++m) {
          const int out = pick_free();
          if (out < 0) return NS_ERR_BUDGET;
          std::vector<const double*> in = states(cur);
          std::vector<double*> wo(n);
          for (int k = 0; k < n; ++k) wo[k] = buf[k][out];
          if ((r = ns_slab_primal_step(G, in.data(), s, wo.data()))) return r;
          cur = out;
        }
        break;
      case NS_OP_STORE:
        if (cur < 0) return NS_ERR_ARG;
        slot_buf[A.b] = cur;
        owned[cur] = 1;
        break;
      case NS_OP_LOAD:
        cur = A.b < 0 ? -1 : slot_buf[A.b];
        break;
      case NS_OP_FREE:
        owned[slot_buf[A.b]] = 0;
        slot_buf[A.b] = -1;
        break;
      case NS_OP_SOURCE: {
        for (int k = 0; k < n; ++k)
          if (cudaMemsetAsync(lc[k], 0, G->c[k]->field * sizeof(double), G->c[k]->st) != cudaSuccess)
            return NS_ERR_CUDA;
        if ((r = ns_objective(co, states(cur)[own], wN, Jbar, lc[own]))) return r;
        if ((r = slab_exchange(G, (void* const*)lc.data(), (int)sizeof(double), 5))) return r;
        break;
      }
      case NS_OP_ADJOINT: {
        std::vector<const double*> w = states(cur);
        if (o->lambda > 0.0) {
          for (int k = 0; k < n; ++k)
            if ((r = ns_growth_sigma1(G->c[k], w[k], sig[k], nullptr)) ||
                (r = ns_add_adjoint_viscosity(G->c[k], sig[k], o->lambda, o->tau, nu[k])))
              return r;
          if ((r = slab_exchange(G, (void* const*)nu.data(), (int)sizeof(float), 1))) return r;
        }
        std::vector<const double*> lin(lc.begin(), lc.end());
        std::vector<const float*> nup(nu.begin(), nu.end());
        if ((r = ns_slab_adjoint_step(G, w.data(), s, lin.data(), o->lambda > 0.0 ? nup.data() : nullptr,
                                      ln.data())))
          return r;
        std::swap(lc, ln);
        if (A.a >= 1) {
          if ((r = ns_objective(co, w[own], wN, Jbar, lc[own]))) return r;
          if ((r = slab_exchange(G, (void* const*)lc.data(), (int)sizeof(double), 5))) return r;
        }
        break;
      }
      default:
        return NS_ERR_ARG;
    }
  }
  return NS_OK;
}

}  // extern "C"
