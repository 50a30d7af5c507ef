// Context object behind the opaque ns_ctx handle of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/ns_adjoint.h"
#include "ns_common.cuh"
#include "ns_kernels.h"

struct ns_sweep_state;

struct ns_ctx {
  ns_params p;
  cudaStream_t st = nullptr;
  ns::GridDesc g;
  ns::Coef<double> cd;
  ns::Coef<float> cf;
  ns::Coef<ns::Dual> cx;
  size_t field = 0;              // elements of one [batch][5][cells] field
  double nu_split[3] = {1.0, 1.0, 1.0};   // added-viscosity factors: rho, rho u, rho E
  int nu_cap = 0;                         // hold nu at the explicit limit (ns_set_viscosity_cap)
  int pipeline = -1;                      // pipelined stride sweeps: 1 on, 0 off, -1 NS_PIPELINE
  // stage buffers of the stage type (double in FP64 mode, float in MIXED mode):
  // float mirrors of w and lambda, stage states W2..W4, two seeds, the stage-product
  // (or RK increment) sum and the seed sum
  static constexpr int NSTAGE = 9;
  void* stage[NSTAGE] = {};
  double* tan[6] = {};           // FP64 buffers of the tangent step, allocated on first use
  double* scratch = nullptr;     // reduction scratch
  size_t scratch_n = 0;
  unsigned* err = nullptr;       // sticky device error word
  size_t ws_bytes = 0;
  bool prof_on = false;          // event pairs around each step's adjoint-stage launches
  size_t prof_used = 0;
  long long prof_launches = 0;   // adjoint-stage launches inside the event pairs
  std::vector<cudaEvent_t> events;
  ns_sweep_state* sweep = nullptr;   // executor state between ns_forward_run and ns_backward_run
  long long sweep_gen = 0;           // forward sweeps started on this context
  long long pending_gen = 0;         // generation of the forward sweep awaiting its backward (0: none)
  double* qbar = nullptr;            // box-mean primitive states [batch][5] (closure features)
  unsigned* ticket = nullptr;        // per-box counters of the single-launch objective
  // the sweep's objective sums on a side stream, concurrent with sigma_1 (their own
  // scratch and counters; forked from and joined to st with events)
  cudaStream_t ost = nullptr;
  cudaEvent_t ofork = nullptr, ojoin = nullptr;
  double* oscratch = nullptr;
  unsigned* oticket = nullptr;
  float* train_scratch = nullptr;    // closure training partials, allocated on first use
  size_t train_scratch_n = 0;
  // bounded box (ns_set_boundaries): the padded grid and its workspace
  ns::BcDesc bc{};
  ns::GridDesc gp{};
  void* bstage[6] = {};              // padded stage type: W1..W4, increment sum, adjoint seed
  double* bd[4] = {};                // padded FP64: state, output, source, transposed product
  double* ba[3] = {};                // FP64: seed, next seed, stage-product sum
  void* bsig = nullptr;              // padded sigma_1 (double in FP64 contexts)
  // the replay context of a pipelined stride sweep (created on first use): the same box
  // and parameters, its own stage buffers and stream; it reports into this context's
  // error word
  ns_ctx* rctx = nullptr;
  unsigned* own_err = nullptr;       // a replay context's own error word (err is its owner's)
  bool owns_stream = false;          // st was created by the library (a replay context)
  bool bounded() const { return bc.inout || bc.walls; }
};

// releases the sweep executor state of a context (defined with the executor)
void ns_sweep_release(ns_ctx* c);

// step variants for the executor (ns_api.cu): optional float mirrors (mixed mode) of
// the input and output states and kept stage states W2..W4 (stage-type buffers)
int ns_i_primal(ns_ctx* c, const double* w, const void* w_mirror, const double* s, double* wo, void* wo_mirror,
                void* const* keep3);
// the objective source of an adjoint step, folded into its last transposed stage
struct ns_obj_src {
  const double* aface;
  const double* ndsc;
  int iL, iR;
};
int ns_i_adjoint(ns_ctx* c, const double* w, const void* w_mirror, const void* const* kept3, const double* s,
                 const double* lam, const void* lam_mirror, const float* nu, double* lo, void* lo_mirror,
                 double* sbar, const double* nud = nullptr, const ns_obj_src* obj = nullptr);
// J_acc += weight J(w) and the gradient factors of the objective source for ns_i_adjoint,
// on the side stream ost after the work enqueued on st so far, in the side stream's own
// scratch and counters (held until the adjoint step has run); ns_i_objective_join makes
// st wait for it
int ns_i_objective_sum_forked(ns_ctx* c, const double* w, double weight, double* J_acc, ns_obj_src* obj);
int ns_i_objective_join(ns_ctx* c);
// ns_mlp_features from the float mirror of w when given (mixed mode; the same bits)
int ns_i_mlp_features(ns_ctx* c, const double* w, const void* w_mirror, float* feat);
// ns_adjoint_energy from the float mirrors of w and lam when both are given (mixed mode)
int ns_i_energy(ns_ctx* c, const double* w, const void* w_mirror, const double* lam, const void* lam_mirror,
                double* E);
// sigma_1 (and its stats when stats != null); with nu != null also the viscosity of the
// sigma_1 rule (nu = lambda sigma_1 [sigma_1 > tau]) with the stability flag
int ns_i_sigma1(ns_ctx* c, const double* w, const void* w_mirror, float* sigma1, double* stats,
                double lambda = 0.0, double tau = 0.0, float* nu = nullptr);
// FP64 contexts: sigma_1 (and with nu != null the rule's viscosity) kept in FP64
int ns_i_sigma1_f64(ns_ctx* c, const double* w, double* sigma1, double* stats, double lambda, double tau,
                    double* nu);
size_t ns_i_stage_bytes(const ns_ctx* c);

namespace ns {
// out2[0] = sum (b - a)^2, out2[1] = sum b^2 over n doubles (FP64, deterministic; uses
// 2 x 296 doubles of scratch)
cudaError_t launch_diff_norms(const double* a, const double* b, size_t n, double* out2, double* scratch,
                              cudaStream_t st);
}  // namespace ns
