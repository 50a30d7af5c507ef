// Shared device-side definitions of the NS stencil kernels (sm_103a).
//
// Tile geometry: a CTA owns TX x TY cell columns of one box and marches a chunk of
// z-planes, keeping a ring of three planes (k-1, k, k+1) of primitive variables with
// a one-cell halo in x and y in shared memory.  Every face flux of the chunk is
// computed once; periodic wrap is resolved when a plane is loaded, so every shared
// position holds a valid cell even when the box is smaller than the tile.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ns {

constexpr int TX = 32;
constexpr int TY = 4;
constexpr int NT = TX * TY;   // threads per CTA
constexpr int SX = TX + 2;    // shared plane width incl. halo
constexpr int SY = TY + 2;
constexpr int SP = SX * SY;   // cells per shared plane

struct GridDesc {
  int nx, ny, nz, batch;
  int kchunk;          // z-planes per CTA
  int nzchunks;        // ceil(nz / kchunk)
  long long plane;     // nx * ny
  long long cells;     // nx * ny * nz  (one box)
};

template <class T>
struct Coef {
  T gamma, gm1, mu, alpha;
  T idx[3];    // 1 / dx_d
  T i4dx[3];   // 1 / (4 dx_d): tangential face gradient = mean of two central diffs
  T hidx[3];   // 1 / (2 dx_d): cell-centred central difference
};

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

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
// error word bits (sticky, OR-ed by kernels, read by ns_last_error)
// ---------------------------------------------------------------------------------
constexpr unsigned ERRBIT_NONFINITE = 1u;
constexpr unsigned ERRBIT_UNSTABLE = 2u;

}  // namespace ns
