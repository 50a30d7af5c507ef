// Shared device-side definitions of the NS stencil kernels (sm_103a).
//
// Tile geometry: a CTA owns TX x TY cell columns of one box (TX = 32 below; both stage
// kernels use 32 x 8, their TY set in their own files) and marches a range of
// z-planes, keeping a ring of three planes (k-1, k, k+1) of primitive variables with
// a one-cell halo in x and y in shared memory.  Every face flux of the range is
// computed once; periodic wrap is resolved when a plane is loaded, so every shared
// position holds a valid cell even when the box is smaller than the tile.
//
// Work split: the CTAs of a launch, as many as the kernel has resident slots on the
// device (occupancy calculator x SMs), are dealt out to the tile columns as evenly as
// integers allow (column c gets floor((c+1)G/C) - floor(cG/C) of the G CTAs), and each
// column's planes are cut into that many ranges whose lengths differ by at most one.
// One wave of CTAs then covers the grid with every SM holding the same number of CTAs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <atomic>
#include <type_traits>
#include <utility>

namespace ns {

// Process-wide count of this library's kernel launches (read by ns_launch_count).
inline std::atomic<unsigned long long> g_launches{0};
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int TX = 32;
constexpr int SX = TX + 2;    // shared plane width incl. halo

struct GridDesc {
  int nx, ny, nz, batch;
  long long plane;     // nx * ny
  long long cells;     // nx * ny * nz  (one box)
  unsigned* dbg_err;   // sticky error word for the bounds checks of debug builds (may be null)
};

constexpr int MIN_PLANES = 4;   // fewest planes per CTA range (bounds the priming share)

// Plane range of this CTA for tiles of TXK x TYK columns (see the file comment).
template <int TXK, int TYK>
__device__ __forceinline__ void march_range(const GridDesc& g, int& b, int& x0, int& y0, int& kz0,
                                            int& kz1) {
  const int ncx = (g.nx + TXK - 1) / TXK, ncy = (g.ny + TYK - 1) / TYK;
  const long long C = (long long)ncx * ncy * g.batch, G = gridDim.x, i = blockIdx.x;
  const int col = (int)(((i + 1) * C - 1) / G);
  const long long s0 = (long long)col * G / C, s1 = (long long)(col + 1) * G / C;
  const long long j = i - s0, m = s1 - s0;
  kz0 = (int)(g.nz * j / m);
  kz1 = (int)(g.nz * (j + 1) / m);
  x0 = (col % ncx) * TXK;
  const int r = col / ncx;
  y0 = (r % ncy) * TYK;
  b = r / ncy;
}

// Launch shape of a plane-marching kernel (see the file comment): the CTA count.  The resident slots come from the occupancy calculator with
// the kernel's dynamic shared memory and are cached per device; the kernel's dynamic
// shared-memory limit is raised once.  The environment variable `env`, when set to a
// positive count, overrides the CTA count.  At least one CTA per tile column, at most
// nz / MIN_PLANES per column.
template <int TXK, int TYK>
struct MarchShape {
  static constexpr int NTK = TXK * TYK;
  int per_dev[16] = {0};
  template <class K>
  cudaError_t get(K kern, size_t smem, const GridDesc& g, const char* env, int& ctas) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int slots = (dev >= 0 && dev < 16) ? per_dev[dev] : 0;
    if (slots == 0) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int per_sm = 0, sms = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTK, smem);
      if (e != cudaSuccess) return e;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      slots = (per_sm > 0 ? per_sm : 1) * sms;
      if (dev >= 0 && dev < 16) per_dev[dev] = slots;
    }
    const long long cols = (long long)((g.nx + TXK - 1) / TXK) * ((g.ny + TYK - 1) / TYK) * g.batch;
    long long n = slots;
    const char* ov = env ? getenv(env) : nullptr;
    if (ov && atoll(ov) > 0) n = atoll(ov);
    const long long most = cols * (g.nz / MIN_PLANES > 1 ? g.nz / MIN_PLANES : 1);
    if (n > most) n = most;
    if (n < cols) n = cols;
    if (n > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
    ctas = (int)n;
    return cudaSuccess;
  }
};

template <class T>
struct Coef {
  T gamma, gm1, mu, alpha;
  T roe_delta;  // Harten's entropy-fix fraction of the Roe sound speed
  int roe;      // 1: Roe dissipation on the convective face flux
  T idx[3];    // 1 / dx_d
  T i4dx[3];   // 1 / (4 dx_d): tangential face gradient = mean of two central diffs
  T hidx[3];   // 1 / (2 dx_d): cell-centred central difference
};

__device__ __forceinline__ int wrap(int i, int n) {
  if (i >= 0 && i < n) return i;
  i %= n;
  return i < 0 ? i + n : i;
}

// ---------------------------------------------------------------------------------
// IEEE-754 binary64 <-> binary32 conversions in integer arithmetic.  GB300 issues
// FP64 instructions at a small fraction of the FP32 rate, so the mixed-precision path
// converts with integer ALU operations instead, from the field layout of the formats
// (sign, biased exponent, fraction):
//   d2f: round to nearest, ties to even; results below the smallest normal float
//        (2^-126) flush to signed zero; overflow gives infinity; NaN stays NaN.
//   f2d: exact for normal floats and zero; subnormal floats flush to signed zero.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned frac_hi = hi & 0xFFFFFu;            // top 20 fraction bits
  if (e == 0x7FF) {                                   // inf / nan
    const bool nan = (frac_hi | lo) != 0u;
    return __uint_as_float(sign | 0x7F800000u | (nan ? 0x00400000u : 0u));
  }
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);          // zero, subnormal, underflow
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  const unsigned fm = (frac_hi << 3) | (lo >> 29);    // 23 fraction bits
  const unsigned rem = lo & 0x1FFFFFFFu;              // 29 dropped bits
  unsigned r = sign | ((unsigned)fe << 23) | fm;
  if (rem > 0x10000000u || (rem == 0x10000000u && (fm & 1u))) r += 1u;   // carry may reach inf
  return __uint_as_float(r);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  if (e == 0xFFu) return __hiloint2double((int)(sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u)), 0);
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// conversions used by the templated kernels: to the compute type / back to FP64
template <class T> __device__ __forceinline__ T cvt(double x);
template <> __device__ __forceinline__ double cvt<double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt<float>(double x) { return d2f(x); }
template <class T> __device__ __forceinline__ T cvt(float x) { return T(x); }
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return f2d(x); }

// ---------------------------------------------------------------------------------
// forward-mode dual number (value, tangent) used to build the tangent kernel from
// the primal one
// ---------------------------------------------------------------------------------
struct Dual {
  double v, d;
  __host__ __device__ __forceinline__ Dual() {}
  __host__ __device__ __forceinline__ Dual(double a) : v(a), d(0.0) {}
  __host__ __device__ __forceinline__ Dual(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) {
  return Dual(a.v * b.v, a.d * b.v + a.v * b.d);
}
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }

template <class T> struct ValueOf { typedef T type; };
template <> struct ValueOf<Dual> { typedef double type; };

__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ double tan_of(Dual a) { return a.d; }

template <class T> __device__ __forceinline__ T one_over(T a) { return T(1) / a; }

// ---------------------------------------------------------------------------------
// Paired FP32 arithmetic (sm_100 family): one instruction does two independent FP32
// operations.  t2 = ((a - b) + c - d) * s for two such expressions at once, with the
// same rounding as the scalar left-to-right evaluation (a - b is fma(b, -1, a)).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

template <class CT>
__device__ __forceinline__ void diff4_pair(CT a1, CT b1, CT c1, CT d1, CT s1, CT a2, CT b2, CT c2, CT d2, CT s2,
                                           CT& r1, CT& r2) {
  if constexpr (std::is_same<CT, float>::value) {
    float2 t = sub2(f2(a1, a2), f2(b1, b2));
    t = __fadd2_rn(t, f2(c1, c2));
    t = sub2(t, f2(d1, d2));
    t = __fmul2_rn(t, f2(s1, s2));
    r1 = t.x;
    r2 = t.y;
  } else {
    r1 = (a1 - b1 + c1 - d1) * s1;
    r2 = (a2 - b2 + c2 - d2) * s2;
  }
}

// ---------------------------------------------------------------------------------
// programmatic dependent launch.  The stencil and per-step diagnostic kernels of the
// sweep go out with programmatic stream serialisation: the next kernel's CTAs may be
// scheduled while the current kernel drains, so the launch latency between dependent
// kernels overlaps the tail of the previous one.  Each such kernel starts with
// pdl_enter(): griddepcontrol.wait blocks until the preceding grid has completed and
// its memory is visible (a no-op for a launch without the attribute), and only then
// does griddepcontrol.launch_dependents release the kernel after it, so every kernel
// still sees all earlier kernels' results.  The dependent grid starts only after every
// CTA of this one has started, so the early launch cannot starve this grid.  NS_PDL=0
// launches without the attribute.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

inline bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("NS_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

// launch k (whose first statement is pdl_enter()) on st with the PDL attribute
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------------
// error word bits (sticky, OR-ed by kernels, read by ns_last_error)
// ---------------------------------------------------------------------------------
constexpr unsigned ERRBIT_NONFINITE = 1u;
constexpr unsigned ERRBIT_UNSTABLE = 2u;
constexpr unsigned ERRBIT_CORRUPT = 4u;
constexpr unsigned ERRBIT_BOUNDS = 8u;

// An added adjoint viscosity v against the explicit stability limit: held at the limit
// where it exceeds it when cap is set; otherwise left, and flagged (NS_ERR_UNSTABLE) when
// above the limit or not finite.
template <class T>
__device__ __forceinline__ T nu_checked(T v, T limit, bool cap, unsigned* err) {
  if (cap && v > limit) return limit;
  if (!(v <= limit)) atomicOr(err, ERRBIT_UNSTABLE);
  return v;
}

// ---------------------------------------------------------------------------------
// Field accesses of the stencil kernels.  A field element is addressed as a base (box,
// plane and component: uniform over the CTA) plus the thread's in-plane offset.  Debug
// builds (NS_DEBUG_BOUNDS) check the element index base + off against the field's
// extent n before every access: an index outside [0, n) sets ERRBIT_BOUNDS in the
// sticky error word and the access is skipped (a load reads zero), so a wrong index
// shows as an error code instead of a memory fault.  Release builds access directly.
// ---------------------------------------------------------------------------------
#ifdef NS_DEBUG_BOUNDS
__device__ __forceinline__ bool dbg_ok(const GridDesc& g, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  if (g.dbg_err) atomicOr(g.dbg_err, ERRBIT_BOUNDS);
  return false;
}
#define NS_LD(g, p, base, off, n)                                                                  \
  (::ns::dbg_ok((g), (long long)(base) + (long long)(off), (long long)(n))                         \
       ? ((p) + (base))[(off)]                                                                     \
       : std::remove_cv_t<std::remove_reference_t<decltype((p)[0])>>(0))
#define NS_ST(g, p, base, off, n, val)                                                             \
  do {                                                                                             \
    if (::ns::dbg_ok((g), (long long)(base) + (long long)(off), (long long)(n))) ((p) + (base))[(off)] = (val); \
  } while (0)
#define NS_IN_BOUNDS(g, i, n) (::ns::dbg_ok((g), (long long)(i), (long long)(n)))
#else
#define NS_IN_BOUNDS(g, i, n) true
#define NS_LD(g, p, base, off, n) (((p) + (base))[(off)])
#define NS_ST(g, p, base, off, n, val) (((p) + (base))[(off)] = (val))
#endif

}  // namespace ns
