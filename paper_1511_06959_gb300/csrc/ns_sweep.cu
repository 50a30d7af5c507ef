// Host runtime of the checkpointed adjoint sweep: the planner (which primal states to
// keep and when to recompute, section "Implementation" of the paper: periodic
// snapshots and segment recomputation; here also binomial checkpointing) and the
// executor that runs a plan on the context's stream with a pool of state buffers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <vector>

#include "../../include/ns_adjoint.h"
#include "ns_ctx.h"

namespace {

// C(s + r, s), saturating far above any step count
double beta(int s, int r) {
  double v = 1.0;
  for (int i = 1; i <= s; ++i) {
    v = v * (double)(r + i) / (double)i;
    if (v > 1e18) return 1e18;
  }
  return v;
}

// first checkpoint offset for reversing l >= 2 steps with s >= 1 free slots: the right
// part keeps s-1 slots and r repetitions, the left part s slots and r-1 repetitions
int revolve_split(int l, int s) {
  int r = 0;
  while (beta(s, r) < (double)l) ++r;
  const double lo = (double)l - beta(s - 1, r);
  const double hi = beta(s, r - 1);
  double m = std::max(1.0, std::min(lo, hi));
  if (m > l - 1) m = l - 1;
  return (int)m;
}

struct Planner {
  std::vector<ns_action> acts;
  std::vector<int> free_slots;
  int next_slot = 0, live = 0, maxlive = 0;
  long long adv = 0;
  std::map<int, int> slot_of;   // step -> slot for stored states

  void emit(int op, int a, int b) {
    acts.push_back(ns_action{op, a, b});
    if (op == NS_OP_ADVANCE) adv += b - a;
  }
  int alloc() {
    int s;
    if (!free_slots.empty()) {
      s = free_slots.back();
      free_slots.pop_back();
    } else {
      s = next_slot++;
    }
    maxlive = std::max(maxlive, ++live);
    return s;
  }
  void store(int step) {
    const int s = alloc();
    slot_of[step] = s;
    emit(NS_OP_STORE, step, s);
  }
  void load(int step) { emit(NS_OP_LOAD, step, step == 0 ? -1 : slot_of.at(step)); }
  void release(int step) {
    if (step == 0) return;
    const int s = slot_of.at(step);
    emit(NS_OP_FREE, step, s);
    slot_of.erase(step);
    free_slots.push_back(s);
    --live;
  }

  void plan_all(int N) {
    for (int n = 0; n < N; ++n) {
      emit(NS_OP_ADVANCE, n, n + 1);
      if (n + 1 < N) store(n + 1);
    }
    emit(NS_OP_SOURCE, N, 0);
    for (int n = N - 1; n >= 0; --n) {
      load(n);
      emit(NS_OP_ADJOINT, n, 0);
      release(n);
    }
  }

  void plan_stride(int N, int k) {
    for (int n = 0; n < N; ++n) {
      if (n > 0 && n % k == 0) store(n);
      emit(NS_OP_ADVANCE, n, n + 1);
    }
    emit(NS_OP_SOURCE, N, 0);
    for (int a = ((N - 1) / k) * k; a >= 0; a -= k) {
      const int b = std::min(a + k, N);
      load(a);
      for (int j = a + 1; j < b; ++j) {
        emit(NS_OP_ADVANCE, j - 1, j);
        store(j);
      }
      for (int n = b - 1; n >= a; --n) {
        load(n);
        emit(NS_OP_ADJOINT, n, 0);
        release(n);
      }
    }
  }

  // reverse steps [a, b) with state a stored and s free slots
  void reverse(int a, int b, int s) {
    if (b - a == 1) {
      load(a);
      emit(NS_OP_ADJOINT, a, 0);
      return;
    }
    if (s == 0) {
      for (int n = b - 1; n >= a; --n) {
        load(a);
        if (n > a) emit(NS_OP_ADVANCE, a, n);
        emit(NS_OP_ADJOINT, n, 0);
      }
      return;
    }
    const int m = a + revolve_split(b - a, s);
    if (!slot_of.count(m)) {
      load(a);
      emit(NS_OP_ADVANCE, a, m);
      store(m);
    }
    reverse(m, b, s - 1);
    release(m);
    reverse(a, m, s);
  }

  void plan_revolve(int N, int S) {
    // the first descent of the recursion is the forward pass: keep its states there
    std::vector<int> chain;
    int a = 0, s = S;
    while (N - a > 1 && s > 0) {
      a += revolve_split(N - a, s);
      chain.push_back(a);
      --s;
    }
    int prev = 0;
    for (int m : chain) {
      emit(NS_OP_ADVANCE, prev, m);
      store(m);
      prev = m;
    }
    emit(NS_OP_ADVANCE, prev, N);
    emit(NS_OP_SOURCE, N, 0);
    reverse(0, N, S);
  }
};

int make_plan(int N, int schedule, int param, Planner& P) {
  if (N < 1) return NS_ERR_ARG;
  switch (schedule) {
    case NS_CKPT_ALL: P.plan_all(N); break;
    case NS_CKPT_STRIDE:
      if (param < 1) return NS_ERR_ARG;
      P.plan_stride(N, param);
      break;
    case NS_CKPT_REVOLVE:
      if (param < 1) return NS_ERR_ARG;
      P.plan_revolve(N, param);
      break;
    default: return NS_ERR_ARG;
  }
  return NS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t state, lam, sig, nu, scal, total;
  int nbuf;
};

Layout layout_for(const ns_ctx* c, int slots_used) {
  Layout L;
  L.nbuf = slots_used + 2;
  L.state = align256(c->field * sizeof(double));
  L.lam = L.state;
  const size_t cellsb = (size_t)c->g.cells * c->g.batch;
  L.sig = align256(cellsb * sizeof(float));
  L.nu = L.sig;
  L.scal = align256((size_t)c->g.batch * sizeof(double) * 2);
  L.total = L.state * L.nbuf + L.lam + L.sig + L.nu + L.scal;
  return L;
}

}  // namespace

extern "C" {

int ns_plan(int nsteps, int schedule, int param, ns_action* out, int max_actions, int* n_actions,
            int* slots_used, long long* advances) {
  Planner P;
  int r = make_plan(nsteps, schedule, param, P);
  if (r) return r;
  if (n_actions) *n_actions = (int)P.acts.size();
  if (slots_used) *slots_used = P.maxlive;
  if (advances) *advances = P.adv;
  if (out) {
    if ((size_t)max_actions < P.acts.size()) return NS_ERR_BUDGET;
    std::copy(P.acts.begin(), P.acts.end(), out);
  }
  return NS_OK;
}

size_t ns_run_arena_bytes(const ns_ctx* c, const ns_run_opts* o) {
  if (!c || !o) return 0;
  Planner P;
  if (make_plan(o->nsteps, o->schedule, o->param, P)) return 0;
  return layout_for(c, P.maxlive).total;
}

int ns_adjoint_run(ns_ctx* c, const double* w0, const double* s, const ns_run_opts* o, void* arena,
                   size_t arena_bytes, double* Jbar, double* lam0, double* sbar, double* energy,
                   double* sigma_stats) {
  if (!c || !w0 || !o || !arena || !Jbar || !lam0 || lam0 == w0) return NS_ERR_ARG;
  if (((uintptr_t)arena & 255) != 0) return NS_ERR_ARG;
  if (!(o->lambda >= 0.0)) return NS_ERR_ARG;
  Planner P;
  int r = make_plan(o->nsteps, o->schedule, o->param, P);
  if (r) return r;
  const Layout L = layout_for(c, P.maxlive);
  if (arena_bytes < L.total) return NS_ERR_BUDGET;
  const int N = o->nsteps;
  const int B = c->g.batch;
  const double wN = 1.0 / N;
  char* base = (char*)arena;
  std::vector<double*> buf(L.nbuf);
  for (int i = 0; i < L.nbuf; ++i) buf[i] = (double*)(base + (size_t)i * L.state);
  char* q = base + (size_t)L.nbuf * L.state;
  double* lamA = (double*)q;
  q += L.lam;
  float* sig = (float*)q;
  q += L.sig;
  float* nu = (float*)q;
  q += L.nu;
  double* jtmp = (double*)q;
  const bool need_sigma = o->lambda > 0.0 || o->record_sigma;
  cudaStream_t st = c->st;
  const size_t fbytes = c->field * sizeof(double);

  double* lam_cur = (N % 2 == 0) ? lam0 : lamA;
  double* lam_nxt = (N % 2 == 0) ? lamA : lam0;
  if (cudaMemsetAsync(lam_cur, 0, fbytes, st) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaMemsetAsync(Jbar, 0, B * sizeof(double), st) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaMemsetAsync(jtmp, 0, 2 * B * sizeof(double), st) != cudaSuccess) return NS_ERR_CUDA;
  if (sbar && cudaMemsetAsync(sbar, 0, fbytes, st) != cudaSuccess) return NS_ERR_CUDA;

  std::vector<int> slot_buf(std::max(P.maxlive, 1), -1);
  std::vector<char> owned(L.nbuf, 0);
  int cur = -1;   // -1: the caller's w0
  int touched = 0;
  auto ptr = [&](int i) -> const double* { return i < 0 ? w0 : buf[i]; };
  auto pick_free = [&]() -> int {
    for (int i = 0; i < L.nbuf; ++i)
      if (!owned[i] && i != cur) return i;
    return -2;
  };

  for (const ns_action& A : P.acts) {
    switch (A.op) {
      case NS_OP_ADVANCE:
        for (int n = A.a; n < A.b; ++n) {
          const int out = pick_free();
          if (out < 0) return NS_ERR_BUDGET;
          if ((r = ns_primal_step(c, ptr(cur), s, buf[out]))) return r;
          if (n + 1 > touched) {
            if ((r = ns_objective(c, buf[out], wN, Jbar, nullptr))) return r;
            touched = n + 1;
          }
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
      case NS_OP_SOURCE:
        if ((r = ns_objective(c, ptr(cur), wN, jtmp, lam_cur))) return r;
        if (o->record_energy && (r = ns_adjoint_energy(c, ptr(cur), lam_cur, energy + (size_t)A.a * B)))
          return r;
        break;
      case NS_OP_ADJOINT: {
        const float* nup = nullptr;
        if (need_sigma) {
          double* stats = o->record_sigma && sigma_stats ? sigma_stats + (size_t)A.a * 2 * B : nullptr;
          if ((r = ns_growth_sigma1(c, ptr(cur), sig, stats))) return r;
          if (o->lambda > 0.0) {
            if ((r = ns_add_adjoint_viscosity(c, sig, o->lambda, o->tau, nu))) return r;
            nup = nu;
          }
        }
        if ((r = ns_adjoint_step(c, ptr(cur), s, lam_cur, nup, lam_nxt, sbar))) return r;
        std::swap(lam_cur, lam_nxt);
        if (A.a >= 1 && (r = ns_objective(c, ptr(cur), wN, jtmp, lam_cur))) return r;
        if (o->record_energy && (r = ns_adjoint_energy(c, ptr(cur), lam_cur, energy + (size_t)A.a * B)))
          return r;
        break;
      }
      default: return NS_ERR_ARG;
    }
  }
  if (lam_cur != lam0 && cudaMemcpyAsync(lam0, lam_cur, fbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NS_ERR_CUDA;
  return NS_OK;
}

}  // extern "C"
