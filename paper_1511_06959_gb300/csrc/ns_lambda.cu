// Choice of the viscosity scaling factor lambda for a given problem.  The paper's
// conclusion leaves this open; its results section tabulates the adjoint sensitivity
// against lambda next to the finite-difference value (too little viscosity: the adjoint
// grows and the sensitivity is wrong; too much: a slowly growing bias; in between a
// range where the sensitivity hardly moves), and section "Energy analysis" asks the
// added viscosity to keep the adjoint energy from growing.  The rule read from these:
// run the stabilised sweep for ascending candidates, fit the growth of the adjoint
// energy over the second half of each backward sweep (beyond the quadratic growth that
// accumulating the objective source alone gives), measure how much the source
// sensitivity moves from each candidate to the next, and take the smallest candidate
// that is damped and on the plateau.
//
// The sweeps and the field norms run on the device (ns_adjoint_run and one FP64
// reduction per candidate); only the energy series, two norms and the sticky error word
// come back to the host, where the fit and the choice are a few hundred flops.
#include <cmath>
#include <cstdint>
#include <limits>
#include <vector>

#include "ns_ctx.h"

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WorkLayout {
  size_t field = 0, energy = 0, jbar = 0, norms = 0, total = 0;
};

WorkLayout work_layout(const ns_ctx* c, int nsteps) {
  WorkLayout L;
  L.field = al256(c->field * sizeof(double));
  L.energy = al256((size_t)(nsteps + 1) * c->g.batch * sizeof(double));
  L.jbar = al256((size_t)c->g.batch * sizeof(double));
  L.norms = al256(2 * sizeof(double));
  L.total = 3 * L.field + L.energy + L.jbar + L.norms;
  return L;
}

// -M times the least-squares slope of ln(E[m] / (N - m + 1)^2) against m, m = 0..M, for
// box b of a [nsteps+1][batch] series: lam^m sums N - m + 1 bounded source terms, so a
// propagator that does not expand the energy keeps the normalised energy bounded and
// only exponential growth makes it rise
double efolds_box(const double* E, int nsteps, int batch, int b) {
  const int M = nsteps / 2;
  std::vector<double> y(M + 1);
  double ybar = 0.0;
  for (int m = 0; m <= M; ++m) {
    const double v = E[(size_t)m * batch + b];
    if (!(v > 0.0) || !std::isfinite(v)) return std::numeric_limits<double>::infinity();
    y[m] = std::log(v) - 2.0 * std::log((double)(nsteps - m + 1));
    ybar += y[m];
  }
  ybar /= (M + 1);
  const double mbar = 0.5 * M;
  double num = 0.0, den = 0.0;
  for (int m = 0; m <= M; ++m) {
    num += (m - mbar) * (y[m] - ybar);
    den += (m - mbar) * (m - mbar);
  }
  return -M * (num / den);
}

// read the sticky error word and clear it (stream-ordered; the caller synchronises)
int take_err(ns_ctx* c, unsigned* h) {
  if (cudaMemcpyAsync(h, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    return NS_ERR_CUDA;
  if (cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->st) != cudaSuccess) return NS_ERR_CUDA;
  return NS_OK;
}

}  // namespace

extern "C" {

int ns_energy_efolds(const double* E, int nsteps, int batch, double* out) {
  if (!E || !out || nsteps < 2 || batch < 1) return NS_ERR_ARG;
  for (int b = 0; b < batch; ++b) out[b] = efolds_box(E, nsteps, batch, b);
  return NS_OK;
}

int ns_lambda_select(int n, const double* efolds, const double* change, double efold_tol, double rel_tol) {
  if (n < 2 || !efolds || !change) return -1;
  for (int i = 0; i + 1 < n; ++i)
    if (efolds[i] <= efold_tol && change[i] <= rel_tol) return i;
  return -1;
}

size_t ns_estimate_work_bytes(const ns_ctx* c, const ns_run_opts* o) {
  if (!c || !o || o->nsteps < 0) return 0;
  return work_layout(c, o->nsteps).total;
}

int ns_estimate_lambda(ns_ctx* c, const double* w0, const double* s, const ns_run_opts* o,
                       const double* lambdas, int n, double efold_tol, double rel_tol, void* arena,
                       size_t arena_bytes, void* work, size_t work_bytes, double* efolds, double* change,
                       int* chosen) {
  if (!c || !w0 || !o || !lambdas || !arena || !work || !efolds || !change || !chosen) return NS_ERR_ARG;
  if (n < 2 || o->nsteps < 2 || ((uintptr_t)work & 255) != 0) return NS_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!(lambdas[i] >= 0.0) || (i > 0 && !(lambdas[i] > lambdas[i - 1]))) return NS_ERR_ARG;
  const WorkLayout L = work_layout(c, o->nsteps);
  if (work_bytes < L.total) return NS_ERR_BUDGET;
  if (arena_bytes < ns_run_arena_bytes(c, o)) return NS_ERR_BUDGET;
  char* q = (char*)work;
  double* lam0 = (double*)q;
  double* sb[2] = {(double*)(q + L.field), (double*)(q + 2 * L.field)};
  double* E = (double*)(q + 3 * L.field);
  double* J = (double*)(q + 3 * L.field + L.energy);
  double* nrm = (double*)(q + 3 * L.field + L.energy + L.jbar);
  const int B = c->g.batch, N = o->nsteps;
  const double nan = std::numeric_limits<double>::quiet_NaN();
  const double inf = std::numeric_limits<double>::infinity();
  for (int i = 0; i < n; ++i) {
    efolds[i] = nan;
    if (i + 1 < n) change[i] = nan;
  }
  *chosen = -1;
  std::vector<double> Eh((size_t)(N + 1) * B), eb(B);
  // the word's bits from before this call are kept apart from the candidates'
  unsigned prior = 0, all = 0;
  int r = take_err(c, &prior);
  if (r) return r;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return NS_ERR_CUDA;
  ns_run_opts oi = *o;
  oi.record_energy = 1;
  oi.record_sigma = 0;
  for (int i = 0; i < n && r == NS_OK; ++i) {
    oi.lambda = lambdas[i];
    double* cur = sb[i & 1];
    r = ns_adjoint_run(c, w0, s, &oi, arena, arena_bytes, J, lam0, cur, E, nullptr);
    if (r) break;
    double hn[2] = {0.0, 0.0};
    unsigned bits = 0;
    if (cudaMemcpyAsync(Eh.data(), E, Eh.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        (i > 0 && (ns::launch_diff_norms(sb[(i - 1) & 1], cur, c->field, nrm, c->scratch, c->st) != cudaSuccess ||
                   cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)) ||
        take_err(c, &bits) != NS_OK || cudaStreamSynchronize(c->st) != cudaSuccess) {
      r = NS_ERR_CUDA;
      break;
    }
    all |= bits;
    ns_energy_efolds(Eh.data(), N, B, eb.data());
    double e = -inf;
    for (int b = 0; b < B; ++b) e = std::isnan(eb[b]) || eb[b] > e ? eb[b] : e;
    // a run that set the sticky word (non-finite values, viscosity past the scheme's
    // stability limit) does not qualify
    efolds[i] = bits ? inf : e;
    if (i > 0) change[i - 1] = hn[1] > 0.0 ? std::sqrt(hn[0]) / std::sqrt(hn[1]) : (hn[0] > 0.0 ? inf : 0.0);
  }
  // give the caller's ns_last_error the union of the bits
  const unsigned keep = prior | all;
  if (keep && (cudaMemcpyAsync(c->err, &keep, sizeof(unsigned), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
               cudaStreamSynchronize(c->st) != cudaSuccess) && !r)
    r = NS_ERR_CUDA;
  if (r) return r;
  *chosen = ns_lambda_select(n, efolds, change, efold_tol, rel_tol);
  return NS_OK;
}

}  // extern "C"
