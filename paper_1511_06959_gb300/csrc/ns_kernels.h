// Internal launch interface between the C-ABI host code and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "ns_common.cuh"

namespace ns {

// Fused Runge-Kutta stage of the primal (see ns_rhs.cu).  With R = R(W) + src:
//   dacc = (dacc_init ? 0 : dacc) + cacc R        increment sum, stage type
//   Wout = base + cout R + cd dacc                 next stage state, stage type
//   wout = (wbase or 0) + widen(dacc + cacc R)     final state, FP64 (when wout != 0)
//   wout_mirror = wout rounded to the stage type    (when wout_mirror != 0)
template <class TIN, class TST>
struct StageArgs {
  const TIN* W;
  const double* Wd;       // tangent of W (Dual instantiation only)
  const TST* base;
  const double* based;
  const double* src;
  const double* srcd;
  TST* dacc;
  double* daccd;
  int dacc_init;
  double cacc;
  TST* Wout;
  double* Woutd;
  double cout;
  double cd;              // Wout also adds cd times the updated increment sum
  const double* wbase;
  const double* wbased;
  double* wout;
  double* woutd;
  TST* wout_mirror;
};

// Fused stage of the discrete adjoint (see ns_adj.cu), a = ca*A:
//   g     = (dR/dw)(W)^T a + L_nu a
//   Gout  = (Gin or 0) + g                              stage-product sum, stage type
//   lam_out = (lam_in or 0) + widen((Gin or 0) + g)     FP64 (when lam_out != 0)
//   Anext = cl*lamf + cg*g + cs*(Gin + g)              next stage seed
//   SBout = (SBin or 0) + a;  sbar += widen((SBin or 0) + a)   source seeds
template <class TIN, class TA, class TST>
struct AdjArgs {
  const TIN* W;
  const TA* A;
  double ca;
  const float* nu;
  const double* nud;      // FP64 nu (FP64 contexts), in place of nu
  double nus[3];          // viscosity factors of the rho, rho u, rho E adjoints
  const TST* lamf;
  const TST* Gin;
  TST* Gout;
  TST* Anext;
  double cl, cg, cs;      // Anext = cl lamf + cg g + cs (Gin + g)
  const double* lam_in;
  double* lam_out;
  TST* lam_out_mirror;    // lam_out rounded to the stage type (when lam_out != 0)
  const TST* SBin;
  TST* SBout;
  double* sbar;
  // objective source folded into the last stage (lam_out != 0): when obj_ndsc != 0,
  // lam_out of the cells of plane columns obj_iL and obj_iR also receives
  // sc (aface[f][v] - [v = 0] N/D), f = z ny + y, (N/D, sc) = obj_ndsc[2b..] (k_obj_sum)
  const double* obj_aface;
  const double* obj_ndsc;
  int obj_iL, obj_iR;
};

template <class CT, class TIN, class TST>
cudaError_t launch_rhs_stage(const GridDesc& g, const Coef<CT>& c, const StageArgs<TIN, TST>& a,
                             cudaStream_t st);

template <class CT, class TIN, class TA, class TST>
cudaError_t launch_adj_stage(const GridDesc& g, const Coef<CT>& c, const AdjArgs<TIN, TA, TST>& a,
                             cudaStream_t st);

// diagnostics and reductions (ns_diag.cu); `scratch` is context workspace of at
// least diag_scratch_doubles(g) doubles, `err` the sticky device error word
size_t diag_scratch_doubles(const GridDesc& g, int nphi);
cudaError_t launch_objective(const GridDesc& g, double gamma, int plane_i, double pt_in,
                             const double* w, double weight, double* J_acc, double* lam,
                             unsigned* err, double* scratch, cudaStream_t st);
// the objective's plane sums and per-face gradient factors alone (k_obj_sum with the
// gradient): J_acc += weight J; *aface, *ndsc receive the factors for an adjoint stage
// that adds the gradient (AdjArgs::obj_*)
cudaError_t launch_objective_sum(const GridDesc& g, double gamma, int plane_i, double pt_in, const double* w,
                                 double weight, double* J_acc, unsigned* err, double* scratch, unsigned* ticket,
                                 cudaStream_t st, const double** aface, const double** ndsc);
// two-launch objective (value in one launch); ticket: batch zero-initialised counters
cudaError_t launch_objective_fast(const GridDesc& g, double gamma, int plane_i, double pt_in, const double* w,
                                   double weight, double* J_acc, double* lam, unsigned* err, double* scratch,
                                   unsigned* ticket, cudaStream_t st, float* lam_mirror = nullptr);
// nu = lam sigma_1 where sigma_1 > tau, else 0, with the stability flag (see k_nu_rule)
struct NuRule {
  float lam, tau, limit;
  float* nu;      // null: no viscosity output
  unsigned* err;
  double lamd, taud, limitd;   // the same rule in FP64 (with nud)
  double* nud;    // FP64 viscosity output (FP64 contexts, with an FP64 sigma_1 output)
  int cap;        // hold nu at the limit instead of flagging it (ns_set_viscosity_cap)
};

// sigma_1 per cell; stats (may be null): [batch][2] = (max, mean), reduced by the last
// block of each box (ticket: per-box counters, zero on entry and on exit); rule (may be
// null): also writes the viscosity of the sigma_1 rule.
// sigma1d (may be null; FP64 contexts): sigma_1 in FP64 in place of the float field,
// with rule->nud the rule's FP64 viscosity.
template <class CT>
cudaError_t launch_sigma1(const GridDesc& g, const Coef<CT>& c, const CT* w, float* sigma1,
                          double* stats, double* scratch, unsigned* ticket, cudaStream_t st,
                          const NuRule* rule = nullptr, double* sigma1d = nullptr);
template <class CT>
cudaError_t launch_label(const GridDesc& g, const Coef<CT>& c, const CT* w, const double* lam, float* acc,
                         cudaStream_t st);
cudaError_t launch_nu_rule(const GridDesc& g, const float* sigma1, double lambda, double tau,
                           double limit_nu, float* nu, unsigned* err, cudaStream_t st, bool cap = false);
cudaError_t launch_nu_rule_f64(const GridDesc& g, const double* sigma1, double lambda, double tau,
                               double limit_nu, double* nu, unsigned* err, cudaStream_t st, bool cap = false);
cudaError_t launch_visc_apply(const GridDesc& g, const double* idx2, const double* split,
                              const float* nu, const double* a, double* out, cudaStream_t st);
cudaError_t launch_energy(const GridDesc& g, double gamma, double dV, const double* w,
                          const double* lam, double* E, double* scratch, unsigned* err,
                          bool fp32_transform, unsigned* ticket, cudaStream_t st);
// The same from the float mirrors of w and lam (mixed precision): the FP32 transform
// reads the rounded values directly, so each cell's term is bit-identical.
cudaError_t launch_energy_mirrors(const GridDesc& g, double gamma, double dV, const float* wf, const float* lamf,
                                  double* E, double* scratch, unsigned* err, unsigned* ticket, cudaStream_t st);
cudaError_t launch_dot(const double* a, const double* phi, int nphi, size_t n, double* out,
                       double* scratch, cudaStream_t st);
cudaError_t launch_combine(const double* theta, const double* phi, int nphi, size_t n,
                           double* s, cudaStream_t st);
cudaError_t launch_max_wave(const GridDesc& g, double gamma, const double* w, double* out,
                            double* scratch, cudaStream_t st);
cudaError_t launch_to_float(const double* in, float* out, size_t n, cudaStream_t st);
cudaError_t launch_scale_boxes(const GridDesc& g, const double* seed, double* field, cudaStream_t st);
cudaError_t launch_dot_boxes(const GridDesc& g, const double* field, int comp, const double* phi,
                             int nphi, double* out, double* scratch, cudaStream_t st);
// doubles of scratch that launch_objective uses for a grid (its partials and plane sums)
size_t objective_scratch_doubles(const GridDesc& g);

// ---- bounded boxes (ns_bc.cu): characteristic inflow/outflow in x, isothermal walls in y
struct BcDesc {
  int inout;          // 1: characteristic inflow at x = 0 and outflow at x = L_x
  int walls;          // 1: isothermal no-slip walls at y = 0 and y = L_y
  double gamma;
  double far[5];      // far-field primitive state (rho, u1, u2, u3, p)
  double wall_e[2];   // internal energy e = c_v T of the bottom and the top wall
};
// one transposed stage's boundary epilogue (see k_bc_adj_epilogue)
struct BcEpilogue {
  const double* A;    // the stage's seed is sa * A (unpadded)
  double sa;
  double nus[3];      // viscosity factors of rho, rho u, rho E
  double i2[3];       // 1 / dx_d^2
  int mode, first, last;
  const double* lam;
  double* G;
  double cl, cg, cs;
  double* a_next;
  double* out;
  double* sbar;
};
long long bc_padded_cells(const GridDesc& g, const BcDesc& bc);
template <class TO, class TI>
cudaError_t launch_bc_embed(const GridDesc& g, const BcDesc& bc, int ncomp, double scale, const TI* src, TO* dst,
                            cudaStream_t st);
template <class TO, class TI>
cudaError_t launch_bc_crop(const GridDesc& g, const BcDesc& bc, int ncomp, const TI* src, TO* dst, cudaStream_t st);
template <class T>
cudaError_t launch_bc_ghosts(const GridDesc& g, const BcDesc& bc, T* W, cudaStream_t st);
template <class CT, class NU>
cudaError_t launch_bc_adj_epilogue(const GridDesc& g, const BcDesc& bc, const BcEpilogue& e, const double* gp,
                                   const CT* W, const NU* nu, cudaStream_t st);

}  // namespace ns
