// Allocation-free variant of the pressure-loss objective (ns_objective_noalloc).
//
// Callers that cannot call cudaMalloc (host frameworks owning all device memory through
// their own pool or quota, or loops that must avoid cudaMalloc's implicit device
// synchronisation) get the objective and its gradient with the reduction scratch in a
// file-scope device array instead of a context workspace.  The array lives on every
// device that loads the library until the process exits.  In host code its name is only
// a host-side stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress and then passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ns_adjoint.h"
#include "ns_common.cuh"
#include "ns_kernels.h"

namespace {

constexpr size_t kScratchDoubles = 32768;   // 256 KiB
constexpr size_t kErrOffset = kScratchDoubles - 8;   // last 64 bytes hold the error word
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_objective_scratch[kScratchDoubles];

std::mutex g_lock;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_on_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NS_ERR_CUDA;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_objective_scratch) != cudaSuccess || !p) return NS_ERR_CUDA;
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return NS_OK;
}

}  // namespace

extern "C" int ns_objective_noalloc(const ns_params* p, void* stream, const double* w, double weight,
                                    double* J_acc, double* lam) {
  if (!p || !w || !J_acc || lam == w) return NS_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->batch < 1 || !(p->gamma > 1.0)) return NS_ERR_ARG;
  // the size limits of ns_create (the kernels index a plane of faces with 32-bit ints)
  if ((long long)p->nx * p->ny > (1LL << 31) || (long long)p->nx * p->ny * p->nz > (1LL << 40))
    return NS_ERR_ARG;
  if (p->plane_i <= -(1 << 30) || p->plane_i >= (1 << 30)) return NS_ERR_ARG;
  ns::GridDesc g{};
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz;
  g.batch = p->batch;
  g.plane = (long long)p->nx * p->ny;
  g.cells = g.plane * p->nz;
  if (ns::objective_scratch_doubles(g) > kErrOffset) return NS_ERR_BUDGET;
  cudaStream_t st = (cudaStream_t)stream;
  // the scratch address is the current device's: the stream must run on that device
  int dev = 0, sdev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) return NS_ERR_CUDA;
  if (sdev != dev) return NS_ERR_ARG;
  double* scratch = nullptr;
  int r = scratch_on_current_device(&scratch);
  if (r) return r;
  // the kernels OR their non-finite flag into this word; nothing reads it (a non-finite
  // objective shows in J_acc itself), so it is never cleared
  unsigned* err = (unsigned*)(scratch + kErrOffset);
  cudaError_t e = ns::launch_objective(g, p->gamma, p->plane_i, p->pt_in, w, weight, J_acc, lam, err,
                                       scratch, st);
  return e == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}
