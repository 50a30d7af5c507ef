// Host runtime of the checkpointed adjoint sweep: the planner (which primal states to
// keep and when to recompute, section "Implementation" of the paper: periodic
// snapshots and segment recomputation; here also binomial checkpointing) and the
// executor that runs a plan on the context's stream with a pool of state buffers.
#include <cuda_runtime.h>
#include <errno.h>
#include <fcntl.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <unistd.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/ns_adjoint.h"
#include "ns_ctx.h"
#include "ns_kernels.h"

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

// Snapshot checksum: sum over the 64-bit words w_i of a state of mix(w_i + (i + 1) K),
// mix the splitmix64 finaliser, mod 2^64.  Integer addition mod 2^64 is exactly
// associative, so the atomic per-block accumulation gives the same value in any order.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_checksum(const unsigned long long* __restrict__ x, size_t n, unsigned long long* out) {
  unsigned long long s = 0ull;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += mix64(x[i] + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void k_checksum_check(const unsigned long long* a, const unsigned long long* b, unsigned* err) {
  if (*a != *b) atomicOr(err, ns::ERRBIT_CORRUPT);
}

// out = checksum of n 64-bit words (zeroed first)
int checksum(ns_ctx* c, const void* x, size_t n, unsigned long long* out) {
  if (cudaMemsetAsync(out, 0, sizeof(unsigned long long), c->st) != cudaSuccess) return NS_ERR_CUDA;
  k_checksum<<<152 * 4, 256, 0, c->st>>>((const unsigned long long*)x, n, out);
  ns::count_launch();
  return cudaGetLastError() == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

// the checksum of x against the stored one; a mismatch sets the corrupt bit
int checksum_verify(ns_ctx* c, const void* x, size_t n, unsigned long long* tmp, const unsigned long long* want) {
  int r = checksum(c, x, n, tmp);
  if (r) return r;
  k_checksum_check<<<1, 1, 0, c->st>>>(tmp, want, c->err);
  ns::count_launch();
  return cudaGetLastError() == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

struct Planner {
  std::vector<ns_action> acts;
  std::vector<int> free_slots;
  int next_slot = 0, live = 0, maxlive = 0;
  long long adv = 0;
  std::map<int, int> slot_of;   // step -> slot for stored states
  // host slots (NS_CKPT_STRIDE_HOST snapshots), a pool of their own
  std::vector<int> free_hslots;
  int next_hslot = 0, hlive = 0, maxhost = 0;
  std::map<int, int> hslot_of;

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

  void hstore(int step) {
    int h;
    if (!free_hslots.empty()) {
      h = free_hslots.back();
      free_hslots.pop_back();
    } else {
      h = next_hslot++;
    }
    maxhost = std::max(maxhost, ++hlive);
    hslot_of[step] = h;
    emit(NS_OP_STORE_HOST, step, h);
  }
  void hload(int step) { emit(NS_OP_LOAD_HOST, step, hslot_of.at(step)); }
  void hfree(int step) {
    const int h = hslot_of.at(step);
    emit(NS_OP_FREE_HOST, step, h);
    hslot_of.erase(step);
    free_hslots.push_back(h);
    --hlive;
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

  // every k-th state in the forward pass, and every state of the last segment, which the
  // backward pass then reverses without replaying it
  void plan_stride(int N, int k) {
    const int alast = ((N - 1) / k) * k;
    for (int n = 0; n < N; ++n) {
      if (n > 0 && (n % k == 0 || n > alast)) store(n);
      emit(NS_OP_ADVANCE, n, n + 1);
    }
    emit(NS_OP_SOURCE, N, 0);
    for (int a = alast; a >= 0; a -= k) {
      const int b = std::min(a + k, N);
      if (a != alast) {
        load(a);
        for (int j = a + 1; j < b; ++j) {
          emit(NS_OP_ADVANCE, j - 1, j);
          store(j);
        }
      }
      for (int n = b - 1; n >= a; --n) {
        load(n);
        emit(NS_OP_ADJOINT, n, 0);
        release(n);
      }
    }
  }

  // plan_stride with the snapshots in host slots: a segment's snapshot comes back into a
  // device slot once, and the host slot is released at once.  The last segment's states,
  // its first one included, stay in device slots from the forward pass.
  void plan_stride_host(int N, int k) {
    const int alast = ((N - 1) / k) * k;
    for (int n = 0; n < N; ++n) {
      if (n > 0 && n >= alast) {
        store(n);
      } else if (n > 0 && n % k == 0) {
        hstore(n);
      }
      emit(NS_OP_ADVANCE, n, n + 1);
    }
    emit(NS_OP_SOURCE, N, 0);
    for (int a = alast; a >= 0; a -= k) {
      const int b = std::min(a + k, N);
      if (a != alast) {
        if (a == 0) {
          load(0);
        } else {
          hload(a);
          store(a);
          hfree(a);
        }
        for (int j = a + 1; j < b; ++j) {
          emit(NS_OP_ADVANCE, j - 1, j);
          store(j);
        }
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
    case NS_CKPT_STRIDE_HOST:
    case NS_CKPT_STRIDE_DISK:
      if (param < 1) return NS_ERR_ARG;
      P.plan_stride_host(N, param);
      break;
    case NS_CKPT_REVOLVE_HOST:
    case NS_CKPT_REVOLVE_DISK: {
      // the revolve plan with every checkpoint slot a host (file) slot: the device keeps
      // only the working states
      if (param < 1) return NS_ERR_ARG;
      Planner D;
      D.plan_revolve(N, param);
      for (ns_action a : D.acts) {
        if (a.op == NS_OP_STORE) a.op = NS_OP_STORE_HOST;
        else if (a.op == NS_OP_LOAD && a.b >= 0) a.op = NS_OP_LOAD_HOST;
        else if (a.op == NS_OP_FREE) a.op = NS_OP_FREE_HOST;
        P.acts.push_back(a);
      }
      P.adv = D.adv;
      P.maxhost = D.maxlive;
      P.maxlive = 0;
      break;
    }
    default: return NS_ERR_ARG;
  }
  return NS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// n bytes between buf and the file at offset off, in as many calls as the kernel needs;
// false on an error or an early end of file
bool file_io(int fd, void* buf, size_t n, long long off, bool write) {
  char* p = (char*)buf;
  while (n > 0) {
    const ssize_t k = write ? pwrite(fd, p, n, (off_t)off) : pread(fd, p, n, (off_t)off);
    if (k < 0 && errno == EINTR) continue;
    if (k <= 0) return false;
    p += k;
    off += k;
    n -= (size_t)k;
  }
  return true;
}

// Arena regions.  mir: two stage-type fields holding float mirrors of consecutive
// states of an ADVANCE run (mixed precision).  lmir: two float mirrors of the adjoint,
// written by the last adjoint stage and kept in step by the objective source, so that
// the next adjoint step needs no conversion (mixed precision).  keep: for stride schedules, one entry of
// four stage-type fields per step of the segment being reversed (the mirror of w^n and
// the stage states W2..W4 computed when the segment was replayed), so that the adjoint
// of a replayed step neither recomputes its stages nor converts its state.
// pool, keep2: a pipelined stride sweep's second set of kept entries and its two sets of
// k-1 replayed states, plus the segment's snapshot for the host tier (the forward pass's
// buffers hold the last segment's).
struct Layout {
  size_t state, lam, sig, nu, scal, feat, stage, mir, lmir, keep, sums, pool, keep2, total;
  int nbuf, nkeep;
};

// NS_PIPELINE=0 (or ns_set_pipeline(ctx, 0)) reverses the stride plan's segments one
// after the other, each replay before its reversal, on the context's stream alone.
bool pipeline_enabled() {
  static const bool on = [] {
    const char* e = getenv("NS_PIPELINE");
    return !(e && e[0] == '0');
  }();
  return on;
}

// A stride sweep of at least two segments on a periodic box, without snapshot checksums,
// with its snapshots in device or host memory (not in a file, whose accesses wait on the
// stream), replays segment i+1 on a second stream while segment i is reversed.
bool pipelined(const ns_ctx* c, int nsteps, int schedule, int param, bool verify) {
  const bool on = c->pipeline < 0 ? pipeline_enabled() : c->pipeline != 0;
  return on && (schedule == NS_CKPT_STRIDE || schedule == NS_CKPT_STRIDE_HOST) && !c->bounded() && !verify &&
         param >= 2 && nsteps - 1 >= param;
}

Layout layout_for(const ns_ctx* c, int slots_used, bool closure, int schedule, int param, int host_slots = 0,
                  bool verify = false, bool pipe = false) {
  // a bounded box forms its stage states inside its own step calls: nothing is kept
  if (c->bounded()) schedule = -1;
  Layout L;
  L.nbuf = slots_used + 2;
  L.state = align256(c->field * sizeof(double));
  L.lam = L.state;
  const size_t cellsb = (size_t)c->g.cells * c->g.batch;
  // sigma_1 and nu: FP64 in FP64 contexts with the sigma_1 rule, float otherwise
  const size_t ssz = c->p.precision == NS_FP64 && !closure ? sizeof(double) : sizeof(float);
  L.sig = align256(cellsb * ssz);
  L.nu = L.sig;
  L.scal = align256((size_t)c->g.batch * sizeof(double) * 2);
  L.feat = closure ? align256(cellsb * 16 * sizeof(float)) : 0;
  L.stage = align256(ns_i_stage_bytes(c));
  L.mir = 2 * L.stage;
  L.lmir = c->p.precision == NS_MIXED ? 2 * L.stage : 0;
  L.nkeep = (schedule == NS_CKPT_STRIDE || schedule == NS_CKPT_STRIDE_HOST || schedule == NS_CKPT_STRIDE_DISK)
                ? param
                : 0;
  L.keep = (size_t)L.nkeep * 4 * L.stage;
  // snapshot checksums: one per device slot and per host slot, and one to verify into
  L.sums = verify ? align256(sizeof(unsigned long long) * (size_t)(slots_used + host_slots + 1)) : 0;
  // a host-tier set also holds the device copy of its segment's snapshot
  L.pool = pipe ? (size_t)2 * (param - 1 + (schedule == NS_CKPT_STRIDE_HOST ? 1 : 0)) * L.state : 0;
  L.keep2 = pipe ? L.keep : 0;
  L.total = L.state * L.nbuf + L.lam + L.sig + L.nu + L.scal + L.feat + L.mir + L.lmir + L.keep + L.sums + L.pool +
            L.keep2;
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
  return layout_for(c, P.maxlive, o->mlp != nullptr, o->schedule, o->param, P.maxhost, o->verify != 0,
                    pipelined(c, o->nsteps, o->schedule, o->param, o->verify != 0))
      .total;
}

size_t ns_run_host_bytes(const ns_ctx* c, const ns_run_opts* o) {
  if (!c || !o || (o->schedule != NS_CKPT_STRIDE_HOST && o->schedule != NS_CKPT_REVOLVE_HOST)) return 0;
  Planner P;
  if (make_plan(o->nsteps, o->schedule, o->param, P)) return 0;
  return (size_t)P.maxhost * align256(c->field * sizeof(double));
}

}  // extern "C"

// Executor state between the forward part of a plan (up to its SOURCE action) and the
// backward part; owned by the context.
struct ns_sweep_state {
  Planner P;
  Layout L;
  ns_run_opts o;
  const double* w0 = nullptr;
  const double* s = nullptr;
  std::vector<double*> buf;
  double* lamA = nullptr;
  float* sig = nullptr;
  float* nu = nullptr;
  bool f64nu = false;                // sigma_1 and nu held in FP64 (the regions hold doubles)
  bool bounded = false;              // a bounded box: every step through the public step calls
  unsigned long long* sums = nullptr; // snapshot checksums (verify): device slots, host slots, scratch
  double* jtmp = nullptr;
  float* feat = nullptr;
  double* Jbar = nullptr;
  std::vector<int> slot_buf;
  std::vector<char> owned;
  int cur = -1;       // -1: the caller's w0
  int touched = 0;
  size_t pos = 0;     // next action
  bool forward_done = false;
  bool obj_forward = true;           // evaluate J(w^n) when the forward pass first reaches n
  bool in_backward = false;
  bool mixed = false;
  char* mir[2] = {nullptr, nullptr};
  void* cur_mirror = nullptr;        // float mirror of the current state, if any
  std::vector<char*> keep;           // [nkeep][4]
  std::vector<char> has_mirror, has_stages;
  int seg = -1;                      // first step of the segment the keep entries belong to
  char* lamf_cur = nullptr;          // float mirror of lam_cur (mixed), valid when lamf_valid
  char* lamf_nxt = nullptr;
  bool lamf_valid = false;
  bool kept_valid(int n) const { return L.nkeep > 0 && seg >= 0 && (n / L.nkeep) * L.nkeep == seg; }
  // NS_CKPT_STRIDE_DISK: the snapshot file and the page-locked staging buffer of one state
  int fd = -1;
  std::string path;
  void* staging = nullptr;
  // pipelined stride sweep: the replay context, the two sets of replayed states and the
  // second set of kept entries, the forward-pass buffer of each stored step, and the
  // events that order the replay stream against the context's stream
  bool pipe = false;
  ns_ctx* rc = nullptr;
  std::vector<double*> pool[2];
  std::vector<char*> keep2;
  std::vector<int> buf_of_step;
  std::vector<int> hslot_of_step;        // host tier: the host slot of each snapshot
  cudaEvent_t ev_fwd = nullptr, ev_rep[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  ~ns_sweep_state() {
    if (fd >= 0) {
      close(fd);
      unlink(path.c_str());
    }
    if (staging) cudaFreeHost(staging);
    for (cudaEvent_t e : {ev_fwd, ev_rep[0], ev_rep[1], ev_free[0], ev_free[1]})
      if (e) cudaEventDestroy(e);
  }
};

void ns_sweep_release(ns_ctx* c) {
  delete c->sweep;
  c->sweep = nullptr;
}

namespace {

// Adjoint step n of the sweep on the context's stream: sigma_1 and the viscosity, the
// objective's plane sums of w^n on the side stream (n >= 1), the four transposed stages
// with the objective source folded in, and the energy.  w: the state w^n; mirror: its
// float mirror or NULL; kept3: its kept stage states, or NULL to recompute them.
int adjoint_at(ns_ctx* c, ns_sweep_state& S, int n, const double* w, const void* mirror, const void* const* kept3,
               double*& lam_cur, double*& lam_nxt, double* sbar, double* energy, double* sigma_stats) {
  const int B = c->g.batch;
  const double wN = 1.0 / S.o.nsteps;
  const bool need_sigma = S.o.lambda > 0.0 || S.o.record_sigma || S.o.mlp;
  int r;
  const float* nup = nullptr;
  const double* nudp = nullptr;
  // the objective of w^n (n >= 1): its plane sums on the side stream, concurrent with
  // sigma_1, its source folded into the last transposed stage of this step
  ns_obj_src obj{};
  if (n >= 1 && (r = ns_i_objective_sum_forked(c, w, wN, S.jtmp, &obj))) return r;
  if (need_sigma && S.f64nu) {
    double* stats = S.o.record_sigma && sigma_stats ? sigma_stats + (size_t)n * 2 * B : nullptr;
    const bool rule = S.o.lambda > 0.0;
    if ((r = ns_i_sigma1_f64(c, w, (double*)S.sig, stats, S.o.lambda, S.o.tau,
                             rule ? (double*)S.nu : nullptr)))
      return r;
    if (rule) nudp = (const double*)S.nu;
  } else if (need_sigma) {
    double* stats = S.o.record_sigma && sigma_stats ? sigma_stats + (size_t)n * 2 * B : nullptr;
    // the sigma_1 rule's viscosity comes out of the same launch as sigma_1
    const bool rule = !S.o.mlp && S.o.lambda > 0.0;
    if ((r = ns_i_sigma1(c, w, mirror, S.sig, stats, S.o.lambda, S.o.tau, rule ? S.nu : nullptr)))
      return r;
    if (S.o.mlp) {
      if ((r = ns_i_mlp_features(c, w, mirror, S.feat))) return r;
      if ((r = ns_mlp_infer(c, S.o.mlp, S.feat, S.sig, S.o.lambda, S.nu))) return r;
      nup = S.nu;
    } else if (rule) {
      nup = S.nu;
    }
  }
  if (n >= 1 && (r = ns_i_objective_join(c))) return r;
  if ((r = ns_i_adjoint(c, w, mirror, kept3, S.s, lam_cur,
                        S.lamf_valid ? S.lamf_cur : nullptr, nup, lam_nxt, S.lamf_nxt, sbar, nudp,
                        n >= 1 ? &obj : nullptr)))
    return r;
  std::swap(lam_cur, lam_nxt);
  std::swap(S.lamf_cur, S.lamf_nxt);
  S.lamf_valid = S.lamf_cur != nullptr;
  if (S.o.record_energy && energy &&
      (r = ns_i_energy(c, w, mirror, lam_cur, S.lamf_valid ? S.lamf_cur : nullptr,
                       energy + (size_t)n * B)))
    return r;
  return NS_OK;
}

// Run actions [S.pos, end) until (not including) the first action with op == stop_op
// (stop_op = 0: to the end).  lam_cur/lam_nxt, sbar, energy, sigma_stats are used by
// the backward part only.
// NVTX range for the phases of a sweep (forward pass, replay, adjoint steps), visible in
// a timeline profiler; without one attached the calls do nothing.
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
};

int run_actions(ns_ctx* c, ns_sweep_state& S, int stop_op, double*& lam_cur, double*& lam_nxt,
                double* sbar, double* energy, double* sigma_stats) {
  const int N = S.o.nsteps;
  const int B = c->g.batch;
  const double wN = 1.0 / N;
  const bool need_sigma = S.o.lambda > 0.0 || S.o.record_sigma || S.o.mlp;
  auto ptr = [&](int i) -> const double* { return i < 0 ? S.w0 : S.buf[i]; };
  auto pick_free = [&]() -> int {
    for (int i = 0; i < S.L.nbuf; ++i)
      if (!S.owned[i] && i != S.cur) return i;
    return -2;
  };
  int r;
  for (; S.pos < S.P.acts.size(); ++S.pos) {
    const ns_action& A = S.P.acts[S.pos];
    if (stop_op && A.op == stop_op) return NS_OK;
    switch (A.op) {
      case NS_OP_ADVANCE: {
        Phase ph(S.in_backward ? "ns replay" : "ns forward");
        for (int n = A.a; n < A.b; ++n) {
          const int out = pick_free();
          if (out < 0) return NS_ERR_BUDGET;
          const int K = S.L.nkeep;
          // the stride plans replay every segment but the last, whose states they keep from
          // the forward pass: its steps keep their stages there
          const bool keep = K > 0 && !S.bounded && (S.in_backward || n >= ((N - 1) / K) * K);
          void* in_m = S.mixed && !S.bounded ? S.cur_mirror : nullptr;
          void* out_m = nullptr;
          void* keep3[3] = {nullptr, nullptr, nullptr};
          if (keep) {
            const int e = n % K;
            if (e == 0 || !S.kept_valid(n)) {
              std::fill(S.has_mirror.begin(), S.has_mirror.end(), 0);
              std::fill(S.has_stages.begin(), S.has_stages.end(), 0);
              S.seg = n - e;
            }
            char** E = &S.keep[(size_t)e * 4];
            if (S.mixed) {
              if (e == 0 || in_m != E[0]) {
                if (ns::launch_to_float(ptr(S.cur), (float*)E[0], c->field, c->st) != cudaSuccess) return NS_ERR_CUDA;
              }
              in_m = E[0];
              S.has_mirror[e] = 1;
              const int e1 = (n + 1) % K;
              if (e1 != 0) {
                out_m = S.keep[(size_t)e1 * 4];
                S.has_mirror[e1] = 1;
              }
            }
            keep3[0] = E[1];
            keep3[1] = E[2];
            keep3[2] = E[3];
            S.has_stages[e] = 1;
          } else if (S.mixed && !S.bounded) {
            out_m = S.mir[(n + 1) & 1];
            if (in_m == out_m) in_m = nullptr;
          }
          if (S.bounded) {
            if ((r = ns_primal_step(c, ptr(S.cur), S.s, S.buf[out]))) return r;
          } else if ((r = ns_i_primal(c, ptr(S.cur), in_m, S.s, S.buf[out], out_m, keep ? keep3 : nullptr))) {
            return r;
          }
          if (n + 1 > S.touched) {
            if (S.obj_forward && (r = ns_objective(c, S.buf[out], wN, S.Jbar, nullptr))) return r;
            S.touched = n + 1;
          }
          S.cur = out;
          S.cur_mirror = out_m;
        }
        break;
      }
      case NS_OP_STORE:
        if (S.cur < 0) return NS_ERR_ARG;
        S.slot_buf[A.b] = S.cur;
        S.owned[S.cur] = 1;
        if (S.sums && (r = checksum(c, S.buf[S.cur], c->field, S.sums + A.b))) return r;
        break;
      case NS_OP_LOAD: {
        S.cur = A.b < 0 ? -1 : S.slot_buf[A.b];
        if (S.sums && A.b >= 0 &&
            (r = checksum_verify(c, S.buf[S.cur], c->field, S.sums + S.P.maxlive + S.P.maxhost, S.sums + A.b)))
          return r;
        const int K = S.L.nkeep;
        S.cur_mirror = (S.mixed && S.in_backward && S.kept_valid(A.a) && S.has_mirror[A.a % K])
                           ? S.keep[(size_t)(A.a % K) * 4]
                           : nullptr;
        break;
      }
      case NS_OP_FREE:
        S.owned[S.slot_buf[A.b]] = 0;
        S.slot_buf[A.b] = -1;
        break;
      case NS_OP_STORE_HOST: {
        // stream-ordered: later kernels that reuse the buffer run after the copy
        if (S.cur < 0 || A.b < 0 || A.b >= S.P.maxhost) return NS_ERR_ARG;
        if (S.sums && (r = checksum(c, S.buf[S.cur], c->field, S.sums + S.P.maxlive + A.b))) return r;
        const size_t nb = c->field * sizeof(double);
        if (S.fd >= 0) {
          // file slot A.b: through the staging buffer, the stream drained before the write
          if (cudaMemcpyAsync(S.staging, S.buf[S.cur], nb, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
              cudaStreamSynchronize(c->st) != cudaSuccess)
            return NS_ERR_CUDA;
          if (!file_io(S.fd, S.staging, nb, (long long)A.b * (long long)S.L.state, true)) return NS_ERR_IO;
          break;
        }
        char* hp = (char*)S.o.host_arena + (size_t)A.b * S.L.state;
        if (cudaMemcpyAsync(hp, S.buf[S.cur], nb, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
          return NS_ERR_CUDA;
        break;
      }
      case NS_OP_LOAD_HOST: {
        if (A.b < 0 || A.b >= S.P.maxhost) return NS_ERR_ARG;
        const int out = pick_free();
        if (out < 0) return NS_ERR_BUDGET;
        const size_t nb = c->field * sizeof(double);
        if (S.fd >= 0) {
          // the staging buffer is free: every earlier copy through it has completed
          if (!file_io(S.fd, S.staging, nb, (long long)A.b * (long long)S.L.state, false)) return NS_ERR_IO;
          if (cudaMemcpyAsync(S.buf[out], S.staging, nb, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
              cudaStreamSynchronize(c->st) != cudaSuccess)
            return NS_ERR_CUDA;
        } else {
          const char* hp = (const char*)S.o.host_arena + (size_t)A.b * S.L.state;
          if (cudaMemcpyAsync(S.buf[out], hp, nb, cudaMemcpyHostToDevice, c->st) != cudaSuccess)
            return NS_ERR_CUDA;
        }
        if (S.sums && (r = checksum_verify(c, S.buf[out], c->field, S.sums + S.P.maxlive + S.P.maxhost,
                                           S.sums + S.P.maxlive + A.b)))
          return r;
        S.cur = out;
        S.cur_mirror = nullptr;
        break;
      }
      case NS_OP_FREE_HOST:
        break;
      case NS_OP_SOURCE:
        if ((r = ns_objective(c, ptr(S.cur), wN, S.jtmp, lam_cur))) return r;
        S.lamf_valid = false;
        if (S.o.record_energy && energy &&
            (r = ns_adjoint_energy(c, ptr(S.cur), lam_cur, energy + (size_t)A.a * B)))
          return r;
        break;
      case NS_OP_ADJOINT: {
        Phase ph("ns adjoint step");
        if (S.bounded) {
          // the public step calls, which pad the box with its ghost layer: sigma_1 and the
          // rule's viscosity, the step, then the objective source of w^n (n >= 1)
          const double* w = ptr(S.cur);
          const float* nup = nullptr;
          const double* nudp = nullptr;
          if (S.o.lambda > 0.0 && S.f64nu) {
            if ((r = ns_growth_sigma1_f64(c, w, (double*)S.sig, nullptr)) ||
                (r = ns_add_adjoint_viscosity_f64(c, (double*)S.sig, S.o.lambda, S.o.tau, (double*)S.nu)))
              return r;
            nudp = (const double*)S.nu;
          } else if (S.o.lambda > 0.0) {
            if ((r = ns_growth_sigma1(c, w, S.sig, nullptr)) ||
                (r = ns_add_adjoint_viscosity(c, S.sig, S.o.lambda, S.o.tau, S.nu)))
              return r;
            nup = S.nu;
          }
          r = nudp ? ns_adjoint_step_f64(c, w, S.s, lam_cur, nudp, lam_nxt, sbar)
                   : ns_adjoint_step(c, w, S.s, lam_cur, nup, lam_nxt, sbar);
          if (r) return r;
          std::swap(lam_cur, lam_nxt);
          if (A.a >= 1 && (r = ns_objective(c, w, wN, S.jtmp, lam_cur))) return r;
          S.lamf_valid = false;
          if (S.o.record_energy && energy && (r = ns_adjoint_energy(c, w, lam_cur, energy + (size_t)A.a * B)))
            return r;
          break;
        }
        const int K = S.L.nkeep;
        const void* mirror = S.mixed ? S.cur_mirror : nullptr;
        const void* kept3[3] = {nullptr, nullptr, nullptr};
        bool kept = false;
        if (S.kept_valid(A.a) && S.has_stages[A.a % K]) {
          char** E = &S.keep[(size_t)(A.a % K) * 4];
          kept3[0] = E[1];
          kept3[1] = E[2];
          kept3[2] = E[3];
          kept = true;
          if (S.mixed) mirror = E[0];
        }
        if ((r = adjoint_at(c, S, A.a, ptr(S.cur), mirror, kept ? kept3 : nullptr, lam_cur, lam_nxt, sbar, energy,
                            sigma_stats)))
          return r;
        break;
      }
      default: return NS_ERR_ARG;
    }
  }
  return NS_OK;
}

// The replay context of c: created on first use with c's parameters and a stream of its
// own, reporting into c's error word; its coefficients are refreshed from c (dt may have
// changed) at every sweep.
int replay_context(ns_ctx* c, ns_ctx** out) {
  if (!c->rctx) {
    cudaStream_t rs = nullptr;
    if (cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking) != cudaSuccess) return NS_ERR_CUDA;
    ns_ctx* r = nullptr;
    const int e = ns_create(&c->p, (void*)rs, &r);
    if (e != NS_OK) {
      cudaStreamDestroy(rs);
      return e;
    }
    r->owns_stream = true;
    r->own_err = r->err;
    r->err = c->err;
    r->g.dbg_err = c->err;
    c->rctx = r;
  }
  ns_ctx* r = c->rctx;
  r->p = c->p;
  r->cd = c->cd;
  r->cf = c->cf;
  r->cx = c->cx;
  *out = r;
  return NS_OK;
}

// The stride plan's backward pass, pipelined.  Segment 0 is the last one, whose states
// and kept stages the forward pass left; segment i >= 1 starts at alast - i k and is
// replayed on the replay context's stream into state set and kept-entry set i % 2 while
// segment i-1 is reversed on the context's stream.  A replay waits until the reversal two
// segments back has released its set (ev_free); a reversal waits for its replay (ev_rep).
// Every launch is the one the sequential plan makes, so the bits are the same.
int run_pipelined(ns_ctx* c, ns_sweep_state& S, double*& lam_cur, double*& lam_nxt, double* sbar, double* energy,
                  double* sigma_stats) {
  const int N = S.o.nsteps, k = S.o.param;
  const int alast = ((N - 1) / k) * k;
  const int nseg = alast / k + 1;
  ns_ctx* rc = S.rc;
  if (S.seg != alast) return NS_ERR_ARG;   // the forward pass keeps the last segment
  // no replay reads a checkpoint before the forward pass and the source are done
  if (cudaEventRecord(S.ev_fwd, c->st) != cudaSuccess || cudaStreamWaitEvent(rc->st, S.ev_fwd, 0) != cudaSuccess)
    return NS_ERR_CUDA;
  const bool host = S.o.schedule == NS_CKPT_STRIDE_HOST;
  auto state_of = [&](int i, int n) -> const double* {
    if (n == 0) return S.w0;
    if (i == 0) return S.buf[S.buf_of_step[n]];
    if (n % k == 0) return host ? S.pool[i % 2][k - 1] : S.buf[S.buf_of_step[n]];
    return S.pool[i % 2][n % k - 1];
  };
  auto entry = [&](int i, int e) -> char** { return (i % 2 == 0 ? &S.keep[0] : &S.keep2[0]) + (size_t)e * 4; };
  auto replay = [&](int i) -> int {
    Phase ph("ns replay");
    const int a = alast - i * k, p = i % 2;
    if (i >= 2 && cudaStreamWaitEvent(rc->st, S.ev_free[p], 0) != cudaSuccess) return NS_ERR_CUDA;
    if (host && a > 0) {
      // the segment's snapshot back from its host slot into the set's last buffer
      const char* hp = (const char*)S.o.host_arena + (size_t)S.hslot_of_step[a] * S.L.state;
      if (cudaMemcpyAsync(S.pool[p][k - 1], hp, c->field * sizeof(double), cudaMemcpyHostToDevice, rc->st) !=
          cudaSuccess)
        return NS_ERR_CUDA;
    }
    const double* w = state_of(i, a);
    void* in_m = nullptr;
    if (S.mixed) {
      in_m = entry(i, 0)[0];
      if (ns::launch_to_float(w, (float*)in_m, c->field, rc->st) != cudaSuccess) return NS_ERR_CUDA;
    }
    for (int e = 0; e < k - 1; ++e) {   // step a + e, into state a + e + 1
      char** E = entry(i, e);
      void* out_m = S.mixed ? entry(i, e + 1)[0] : nullptr;
      void* keep3[3] = {E[1], E[2], E[3]};
      double* wo = S.pool[p][e];
      const int r = ns_i_primal(rc, w, in_m, S.s, wo, out_m, keep3);
      if (r) return r;
      w = wo;
      in_m = out_m;
    }
    return cudaEventRecord(S.ev_rep[p], rc->st) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
  };
  auto reverse = [&](int i) -> int {
    Phase ph("ns adjoint step");
    const int a = alast - i * k, b = std::min(a + k, N), p = i % 2;
    if (i >= 1 && cudaStreamWaitEvent(c->st, S.ev_rep[p], 0) != cudaSuccess) return NS_ERR_CUDA;
    for (int n = b - 1; n >= a; --n) {
      const int e = n - a;
      char** E = entry(i, e);
      // the replay forms the stages of every step but the segment's last one
      const bool kept = i == 0 ? S.has_stages[e] != 0 : e < k - 1;
      const bool has_m = i == 0 ? S.has_mirror[e] != 0 : true;
      const void* kept3[3] = {E[1], E[2], E[3]};
      const void* mirror = S.mixed && has_m ? E[0] : nullptr;
      const int r = adjoint_at(c, S, n, state_of(i, n), mirror, kept ? kept3 : nullptr, lam_cur, lam_nxt, sbar,
                               energy, sigma_stats);
      if (r) return r;
    }
    return cudaEventRecord(S.ev_free[p], c->st) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
  };
  int r;
  for (int i = 0; i < nseg; ++i) {
    if (i + 1 < nseg && (r = replay(i + 1))) return r;
    if ((r = reverse(i))) return r;
  }
  S.pos = S.P.acts.size();
  return NS_OK;
}

}  // namespace

extern "C" {

static int forward_run_impl(ns_ctx* c, const double* w0, const double* s, const ns_run_opts* o, void* arena,
                            size_t arena_bytes, double* Jbar, bool objective_in_forward) {
  if (!c || !w0 || !o || !arena || !Jbar) return NS_ERR_ARG;
  // bounded boxes: no learned closure and no sigma_1 statistics (their sigma_1 comes
  // cropped from the padded box)
  if (c->bounded() && (o->mlp || o->record_sigma)) return NS_ERR_ARG;
  if (((uintptr_t)arena & 255) != 0) return NS_ERR_ARG;
  if (!(o->lambda >= 0.0)) return NS_ERR_ARG;
  ns_sweep_release(c);
  c->pending_gen = 0;
  ns_sweep_state* S = new ns_sweep_state();
  int r = make_plan(o->nsteps, o->schedule, o->param, S->P);
  if (r) {
    delete S;
    return r;
  }
  S->pipe = pipelined(c, o->nsteps, o->schedule, o->param, o->verify != 0);
  S->L = layout_for(c, S->P.maxlive, o->mlp != nullptr, o->schedule, o->param, S->P.maxhost, o->verify != 0,
                    S->pipe);
  if (arena_bytes < S->L.total) {
    delete S;
    return NS_ERR_BUDGET;
  }
  if ((o->schedule == NS_CKPT_STRIDE_HOST || o->schedule == NS_CKPT_REVOLVE_HOST) && S->P.maxhost > 0 &&
      (!o->host_arena || o->host_bytes < (size_t)S->P.maxhost * S->L.state)) {
    delete S;
    return NS_ERR_BUDGET;
  }
  if (o->schedule == NS_CKPT_STRIDE_DISK || o->schedule == NS_CKPT_REVOLVE_DISK) {
    if (!o->disk_path || !o->disk_path[0]) {
      delete S;
      return NS_ERR_ARG;
    }
    S->path = o->disk_path;
    S->fd = open(S->path.c_str(), O_RDWR | O_CREAT | O_TRUNC, 0600);
    if (S->fd < 0) {
      delete S;
      return NS_ERR_IO;
    }
    if (cudaMallocHost(&S->staging, c->field * sizeof(double)) != cudaSuccess) {
      S->staging = nullptr;
      delete S;
      return NS_ERR_CUDA;
    }
  }
  S->o = *o;
  S->w0 = w0;
  S->s = s;
  S->Jbar = Jbar;
  S->obj_forward = objective_in_forward;
  char* base = (char*)arena;
  S->buf.resize(S->L.nbuf);
  for (int i = 0; i < S->L.nbuf; ++i) S->buf[i] = (double*)(base + (size_t)i * S->L.state);
  char* q = base + (size_t)S->L.nbuf * S->L.state;
  S->lamA = (double*)q;
  q += S->L.lam;
  S->sig = (float*)q;
  q += S->L.sig;
  S->nu = (float*)q;
  q += S->L.nu;
  S->jtmp = (double*)q;
  q += S->L.scal;
  S->feat = S->L.feat ? (float*)q : nullptr;
  q += S->L.feat;
  S->mir[0] = q;
  S->mir[1] = q + S->L.stage;
  q += S->L.mir;
  S->lamf_cur = S->L.lmir ? q : nullptr;
  S->lamf_nxt = S->L.lmir ? q + S->L.stage : nullptr;
  q += S->L.lmir;
  S->keep.resize((size_t)S->L.nkeep * 4);
  for (size_t i = 0; i < S->keep.size(); ++i) S->keep[i] = q + i * S->L.stage;
  q += S->L.keep;
  S->sums = S->L.sums ? (unsigned long long*)q : nullptr;
  q += S->L.sums;
  if (S->pipe) {
    const int per_set = o->param - 1 + (o->schedule == NS_CKPT_STRIDE_HOST ? 1 : 0);
    for (int p = 0; p < 2; ++p)
      for (int i = 0; i < per_set; ++i) {
        S->pool[p].push_back((double*)q);
        q += S->L.state;
      }
    S->keep2.resize(S->keep.size());
    for (size_t i = 0; i < S->keep2.size(); ++i) S->keep2[i] = q + i * S->L.stage;
    q += S->L.keep2;
    int e = replay_context(c, &S->rc);
    for (cudaEvent_t* ev : {&S->ev_fwd, &S->ev_rep[0], &S->ev_rep[1], &S->ev_free[0], &S->ev_free[1]})
      if (e == NS_OK && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) e = NS_ERR_CUDA;
    if (e != NS_OK) {
      delete S;
      return e;
    }
  }
  S->has_mirror.assign(S->L.nkeep, 0);
  S->has_stages.assign(S->L.nkeep, 0);
  S->mixed = c->p.precision == NS_MIXED;
  S->f64nu = !S->mixed && o->mlp == nullptr;
  S->bounded = c->bounded();
  S->slot_buf.assign(std::max(S->P.maxlive, 1), -1);
  S->owned.assign(S->L.nbuf, 0);
  c->sweep = S;
  const int B = c->g.batch;
  if (cudaMemsetAsync(Jbar, 0, B * sizeof(double), c->st) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaMemsetAsync(S->jtmp, 0, 2 * B * sizeof(double), c->st) != cudaSuccess) return NS_ERR_CUDA;
  double* dummy = nullptr;
  r = run_actions(c, *S, NS_OP_SOURCE, dummy, dummy, nullptr, nullptr, nullptr);
  if (r) return r;
  S->forward_done = true;
  c->pending_gen = ++c->sweep_gen;
  return NS_OK;
}

int ns_forward_run(ns_ctx* c, const double* w0, const double* s, const ns_run_opts* o, void* arena,
                   size_t arena_bytes, double* Jbar) {
  return forward_run_impl(c, w0, s, o, arena, arena_bytes, Jbar, true);
}

int ns_backward_run(ns_ctx* c, double* lam0, double* sbar, double* energy, double* sigma_stats) {
  if (!c || !lam0 || !c->sweep || !c->sweep->forward_done) return NS_ERR_ARG;
  ns_sweep_state& S = *c->sweep;
  if (lam0 == S.w0 || (sbar && (sbar == lam0 || sbar == S.w0))) return NS_ERR_ARG;
  const size_t fbytes = c->field * sizeof(double);
  const int N = S.o.nsteps;
  double* lam_cur = (N % 2 == 0) ? lam0 : S.lamA;
  double* lam_nxt = (N % 2 == 0) ? S.lamA : lam0;
  if (cudaMemsetAsync(lam_cur, 0, fbytes, c->st) != cudaSuccess) return NS_ERR_CUDA;
  if (sbar && cudaMemsetAsync(sbar, 0, fbytes, c->st) != cudaSuccess) return NS_ERR_CUDA;
  S.lamf_valid = false;
  S.forward_done = false;   // a plan is reversed once
  c->pending_gen = 0;
  S.in_backward = true;
  int r;
  if (S.pipe) {
    // the forward pass's buffer of every stored step (nothing is freed before the source)
    S.buf_of_step.assign(N, -1);
    S.hslot_of_step.assign(N, -1);
    for (size_t i = 0; i < S.pos && i < S.P.acts.size(); ++i) {
      const ns_action& A = S.P.acts[i];
      if (A.op == NS_OP_STORE) S.buf_of_step[A.a] = S.slot_buf[A.b];
      if (A.op == NS_OP_STORE_HOST) S.hslot_of_step[A.a] = A.b;
    }
    // the source at step N, then the segments (the plan's remaining actions describe the
    // same steps in sequence)
    r = run_actions(c, S, NS_OP_ADJOINT, lam_cur, lam_nxt, sbar, energy, sigma_stats);
    if (!r) r = run_pipelined(c, S, lam_cur, lam_nxt, sbar, energy, sigma_stats);
  } else {
    r = run_actions(c, S, 0, lam_cur, lam_nxt, sbar, energy, sigma_stats);
  }
  if (r) return r;
  if (lam_cur != lam0 &&
      cudaMemcpyAsync(lam0, lam_cur, fbytes, cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
    return NS_ERR_CUDA;
  ns_sweep_release(c);
  return NS_OK;
}

int ns_adjoint_run(ns_ctx* c, const double* w0, const double* s, const ns_run_opts* o, void* arena,
                   size_t arena_bytes, double* Jbar, double* lam0, double* sbar, double* energy,
                   double* sigma_stats) {
  if (!c || !w0 || !o || !arena || !Jbar || !lam0 || lam0 == w0) return NS_ERR_ARG;
  // The backward pass evaluates J(w^n) for every n = N..1 (for the objective source), so
  // the forward pass skips its own evaluations and Jbar is taken from the backward sums.
  int r = forward_run_impl(c, w0, s, o, arena, arena_bytes, Jbar, false);
  if (r) return r;
  const double* jtmp = c->sweep->jtmp;
  if ((r = ns_backward_run(c, lam0, sbar, energy, sigma_stats))) return r;
  return cudaMemcpyAsync(Jbar, jtmp, (size_t)c->g.batch * sizeof(double), cudaMemcpyDeviceToDevice, c->st) ==
                 cudaSuccess
             ? NS_OK
             : NS_ERR_CUDA;
}

long long ns_sweep_generation(const ns_ctx* c) { return c ? c->pending_gen : 0; }

int ns_set_pipeline(ns_ctx* c, int on) {
  if (!c) return NS_ERR_ARG;
  c->pipeline = on ? 1 : 0;
  return NS_OK;
}

// One ns_adjoint_run recorded as a CUDA graph: the executable graph, the context whose
// stream replays it, and the kernel launches it holds.
struct ns_graph {
  ns_ctx* c = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
};

int ns_adjoint_run_capture(ns_ctx* c, const double* w0, const double* s, const ns_run_opts* o, void* arena,
                           size_t arena_bytes, double* Jbar, double* lam0, double* sbar, double* energy,
                           double* sigma_stats, ns_graph** out) {
  if (!out) return NS_ERR_ARG;
  *out = nullptr;
  if (!c || !o) return NS_ERR_ARG;
  // the host and disk tiers copy through host memory (and the disk tier waits on the
  // stream): not a graph
  if (o->schedule == NS_CKPT_STRIDE_HOST || o->schedule == NS_CKPT_STRIDE_DISK ||
      o->schedule == NS_CKPT_REVOLVE_HOST || o->schedule == NS_CKPT_REVOLVE_DISK)
    return NS_ERR_ARG;
  // capture on a stream of our own (the legacy default stream cannot be captured); the
  // context's side stream joins the capture through the sweep's fork and join events
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return NS_ERR_CUDA;
  cudaStream_t st = c->st;
  c->st = cs;
  const unsigned long long k0 = ns::g_launches.load(std::memory_order_relaxed);
  int r = NS_OK;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    r = NS_ERR_CUDA;
  } else {
    r = ns_adjoint_run(c, w0, s, o, arena, arena_bytes, Jbar, lam0, sbar, energy, sigma_stats);
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (r == NS_OK && e != cudaSuccess) r = NS_ERR_CUDA;
  }
  const long long kernels = (long long)(ns::g_launches.load(std::memory_order_relaxed) - k0);
  c->st = st;
  if (r != NS_OK) ns_sweep_release(c);   // a sweep cut short by an error is not reversed later
  cudaGraphExec_t exec = nullptr;
  if (r == NS_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    exec = nullptr;
    r = NS_ERR_CUDA;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  cudaGetLastError();   // clear the runtime's last error after a refused capture
  if (r != NS_OK) return r;
  *out = new ns_graph{c, exec, kernels};
  return NS_OK;
}

int ns_graph_launch(ns_graph* gr) {
  if (!gr) return NS_ERR_ARG;
  return cudaGraphLaunch(gr->exec, gr->c->st) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

long long ns_graph_kernels(const ns_graph* gr) { return gr ? gr->kernels : -1; }

void ns_graph_destroy(ns_graph* gr) {
  if (!gr) return;
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  delete gr;
}

}  // extern "C"
