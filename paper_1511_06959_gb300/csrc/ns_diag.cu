// Objective, growth matrix sigma_1, adjoint viscosity, adjoint energy and FP64
// reductions.  Every reduction is deterministic: fixed grid, fixed per-thread order,
// a shared-memory tree per block, then one block combines the block partials.
#include <math.h>

#include "ns_common.cuh"
#include "ns_kernels.h"

namespace ns {

namespace {

constexpr int RB = 256;      // threads per reduction block
constexpr int RG = 296;      // blocks per reduced quantity (2 x 148, fixed for determinism)
constexpr int RGS = 1184;    // blocks of the streaming field reductions (fixed for determinism)
constexpr int OB = 64;       // threads per block of the objective face kernels

struct AddOp {
  template <class T>
  __device__ T operator()(T a, T b) const { return a + b; }
};
struct MaxOp {
  template <class T>
  __device__ T operator()(T a, T b) const { return fmax(a, b); }
};

// Butterfly reduction over the 32 lanes of a warp (every lane gets the result); the
// order of the operations is fixed, so results are bitwise reproducible.
template <class T, class Op>
__device__ __forceinline__ T warp_reduce(T v, Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block reduction (blockDim.x a power-of-two multiple of 32, at most 1024): each warp
// reduces its lanes in TW, the warp results are widened to double and reduced by the
// first warp in FP64; every thread returns the result.  sh holds >= 32 doubles.  TW =
// float serves maxima (exact in any type); sums are reduced in double.
template <class TW, class Op>
__device__ __forceinline__ double block_reduce(TW v, double* sh, Op op) {
  v = warp_reduce(v, op);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();                 // sh may still be read by a previous reduction
  if (lane == 0) sh[wid] = (double)v;
  __syncthreads();
  if (wid == 0) {
    double x = lane < nw ? sh[lane] : 0.0;
    for (int o = nw >> 1; o > 0; o >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) sh[0] = x;
  }
  __syncthreads();
  return sh[0];
}

// ---------------------------------------------------------------------------------
// pressure-loss objective, Eq. (e:pressure_loss): per-face terms over a grid of
// blocks, block partials, one block per box for the final quotient, then the
// gradient scatter onto the two plane columns
// ---------------------------------------------------------------------------------
struct FaceState {
  double r, u[3], uu, p;
};

__device__ __forceinline__ FaceState face_state(const double* __restrict__ w, size_t box, long long cells,
                                                size_t row, int iL, int iR, double gm1) {
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v] = 0.5 * (w[box + v * cells + row + iL] + w[box + v * cells + row + iR]);
  FaceState f;
  f.r = q[0];
  const double ir = 1.0 / q[0];
  f.u[0] = q[1] * ir;
  f.u[1] = q[2] * ir;
  f.u[2] = q[3] * ir;
  f.uu = f.u[0] * f.u[0] + f.u[1] * f.u[1] + f.u[2] * f.u[2];
  f.p = gm1 * (q[4] - 0.5 * f.r * f.uu);
  return f;
}

__device__ __forceinline__ double pt_factor(double B, double ex) {
  // B^(gamma/(gamma-1)).  gamma = 1.4 gives the exponent 7/2, which the double
  // quotient 1.4/0.4 misses by one ulp: within 1e-12 of 3.5 the closed form B^3 sqrt(B)
  // is used (it differs from pow(B, 1.4/0.4) by about 1e-16 relative and costs a
  // fraction of a double-precision pow)
  return fabs(ex - 3.5) < 1e-12 ? B * B * B * sqrt(B) : pow(B, ex);
}

__global__ void __launch_bounds__(OB) k_obj_partial(GridDesc g, double gamma, int i0, double pt_in,
                                                    const double* __restrict__ w, double* partial) {
  __shared__ double sh[OB];
  const int b = blockIdx.y;
  const int nf = g.ny * g.nz;
  const int iL = wrap(i0 - 1, g.nx), iR = wrap(i0, g.nx);
  const size_t box = (size_t)b * 5 * g.cells;
  const double gm1 = gamma - 1.0, ex = gamma / gm1;
  double N = 0.0, D = 0.0;
  for (int f = blockIdx.x * OB + threadIdx.x; f < nf; f += gridDim.x * OB) {
    const FaceState F = face_state(w, box, g.cells, (size_t)f * g.nx, iL, iR, gm1);
    const double pt = F.p * pt_factor(1.0 + 0.5 * gm1 * F.r * F.uu / (gamma * F.p), ex);
    N += F.r * (pt_in - pt);
    D += F.r;
  }
  N = block_reduce(N, sh, AddOp());
  D = block_reduce(D, sh, AddOp());
  if (threadIdx.x == 0) {
    partial[((size_t)b * 2 + 0) * gridDim.x + blockIdx.x] = N;
    partial[((size_t)b * 2 + 1) * gridDim.x + blockIdx.x] = D;
  }
}

__global__ void __launch_bounds__(RB) k_obj_final(int nblk, double pt_in, double weight, double* partial,
                                                  double* nd, double* J_acc, unsigned* err) {
  __shared__ double sh[RB];
  const int b = blockIdx.x;
  double N = 0.0, D = 0.0;
  for (int i = threadIdx.x; i < nblk; i += RB) {
    N += partial[((size_t)b * 2 + 0) * nblk + i];
    D += partial[((size_t)b * 2 + 1) * nblk + i];
  }
  N = block_reduce(N, sh, AddOp());
  D = block_reduce(D, sh, AddOp());
  if (threadIdx.x == 0) {
    const double J = N / (D * pt_in);
    if (!isfinite(J)) atomicOr(err, ERRBIT_NONFINITE);
    J_acc[b] += weight * J;
    nd[2 * b] = N;
    nd[2 * b + 1] = D;
  }
}

// dJ/dw_f = [d(rho_f (pt_in - pt_f))/dw_f - (N/D) e_0] / (D pt_in), split 1/2 : 1/2
__global__ void __launch_bounds__(OB) k_obj_grad(GridDesc g, double gamma, int i0, double pt_in,
                                                 double weight, const double* __restrict__ w,
                                                 const double* nd, double* lam) {
  const int b = blockIdx.y;
  const int nf = g.ny * g.nz;
  const int iL = wrap(i0 - 1, g.nx), iR = wrap(i0, g.nx);
  const size_t box = (size_t)b * 5 * g.cells;
  const double gm1 = gamma - 1.0, ex = gamma / gm1;
  const double N = nd[2 * b], D = nd[2 * b + 1];
  const double NoD = N / D;
  const double sc = 0.5 * weight / (D * pt_in);
  for (int f = blockIdx.x * OB + threadIdx.x; f < nf; f += gridDim.x * OB) {
    const size_t row = (size_t)f * g.nx;
    const FaceState F = face_state(w, box, g.cells, row, iL, iR, gm1);
    const double r = F.r, ir = 1.0 / r, uu = F.uu, p = F.p;
    const double B = 1.0 + 0.5 * gm1 * r * uu / (gamma * p);
    const double pt = p * pt_factor(B, ex);
    // derivatives of pt in primitive variables (rho, u, p)
    const double dr = pt * uu / (2.0 * p * B);
    const double dp = pt / p * (1.0 - r * uu / (2.0 * p * B));
    double du[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) du[k] = pt * r * F.u[k] / (p * B);
    // chain to conservative variables through dq/dw
    double dw[5];
    dw[0] = dr - (F.u[0] * du[0] + F.u[1] * du[1] + F.u[2] * du[2]) * ir + 0.5 * gm1 * uu * dp;
#pragma unroll
    for (int k = 0; k < 3; ++k) dw[1 + k] = du[k] * ir - gm1 * F.u[k] * dp;
    dw[4] = gm1 * dp;
    double gv[5];
    gv[0] = ((pt_in - pt) - r * dw[0] - NoD) * sc;
#pragma unroll
    for (int v = 1; v < 5; ++v) gv[v] = -r * dw[v] * sc;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      lam[box + v * g.cells + row + iL] += gv[v];
      lam[box + v * g.cells + row + iR] += gv[v];
    }
  }
}

// Objective in two launches.  k_obj_sum: every CTA sums its faces' value terms and,
// when the gradient is asked for, stores for each face the N/D-independent part a_v
// of dJ/dw_f = sc (a_v - [v = 0] N/D), sc = weight / (2 D pt_in) (all FP64: the terms
// p_t,in - p_t and a_0 - N/D cancel).  The last CTA to finish (ticket after a memory
// fence) reduces the partials in a fixed order, forms J and stores (N/D, sc);
// k_obj_scatter then adds the gradient to the two plane columns.
constexpr int OMB = 64;

__global__ void __launch_bounds__(OMB) k_obj_sum(GridDesc g, double gamma, int i0, double pt_in,
                                                 const double* __restrict__ w, double weight, double* J_acc,
                                                 bool want_grad, unsigned* err, double* partial,
                                                 double* aface, double* ndsc, unsigned* ticket) {
  pdl_enter();
  __shared__ double sh[OMB];
  __shared__ bool last;
  const int b = blockIdx.y;
  const int nf = g.ny * g.nz;
  const int iL = wrap(i0 - 1, g.nx), iR = wrap(i0, g.nx);
  const size_t box = (size_t)b * 5 * g.cells;
  const double gm1 = gamma - 1.0, ex = gamma / gm1;
  double N = 0.0, D = 0.0;
  for (int f = blockIdx.x * OMB + threadIdx.x; f < nf; f += gridDim.x * OMB) {
    const FaceState F = face_state(w, box, g.cells, (size_t)f * g.nx, iL, iR, gm1);
    const double r = F.r, p = F.p, uu = F.uu;
    const double ip = 1.0 / p;
    const double B = 1.0 + 0.5 * gm1 / gamma * r * uu * ip;
    const double pt = p * pt_factor(B, ex);
    N += r * (pt_in - pt);
    D += r;
    if (want_grad) {
      const double ir = 1.0 / r, iB = 1.0 / B;
      const double ptpB = pt * ip * iB;             // pt / (p B)
      const double dr = 0.5 * uu * ptpB;
      const double dp = pt * ip - 0.5 * r * uu * ip * ptpB;
      double du[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) du[k] = r * F.u[k] * ptpB;
      double* A = aface + ((size_t)b * nf + f) * 5;
      A[0] = (pt_in - pt) - r * (dr - (F.u[0] * du[0] + F.u[1] * du[1] + F.u[2] * du[2]) * ir + 0.5 * gm1 * uu * dp);
#pragma unroll
      for (int k = 0; k < 3; ++k) A[1 + k] = -r * (du[k] * ir - gm1 * F.u[k] * dp);
      A[4] = -r * gm1 * dp;
    }
  }
  N = block_reduce(N, sh, AddOp());
  D = block_reduce(D, sh, AddOp());
  if (threadIdx.x == 0) {
    partial[((size_t)b * 2 + 0) * gridDim.x + blockIdx.x] = N;
    partial[((size_t)b * 2 + 1) * gridDim.x + blockIdx.x] = D;
    __threadfence();
    last = atomicAdd(&ticket[b], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  N = 0.0;
  D = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += OMB) {
    N += partial[((size_t)b * 2 + 0) * gridDim.x + i];
    D += partial[((size_t)b * 2 + 1) * gridDim.x + i];
  }
  N = block_reduce(N, sh, AddOp());
  D = block_reduce(D, sh, AddOp());
  if (threadIdx.x == 0) {
    const double J = N / (D * pt_in);
    if (!isfinite(J)) atomicOr(err, ERRBIT_NONFINITE);
    J_acc[b] += weight * J;
    ndsc[2 * b] = N / D;
    ndsc[2 * b + 1] = 0.5 * weight / (D * pt_in);
    ticket[b] = 0u;
  }
}

__global__ void k_obj_scatter(GridDesc g, int i0, const double* __restrict__ aface, const double* __restrict__ ndsc,
                              double* __restrict__ lam, float* __restrict__ lamf) {
  pdl_enter();
  const int nf = g.ny * g.nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nf * g.batch) return;
  const int b = (int)(t / nf), f = (int)(t - (long long)b * nf);
  const int iL = wrap(i0 - 1, g.nx), iR = wrap(i0, g.nx);
  const size_t box = (size_t)b * 5 * g.cells, row = (size_t)f * g.nx;
  const double NoD = ndsc[2 * b], sc = ndsc[2 * b + 1];
  const double* A = aface + ((size_t)b * nf + f) * 5;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double gd = sc * (A[v] - (v == 0 ? NoD : 0.0));
    const size_t oL = box + v * g.cells + row + iL, oR = box + v * g.cells + row + iR;
    lam[oL] += gd;
    if (lamf) lamf[oL] = d2f(lam[oL]);
    lam[oR] += gd;
    if (lamf) lamf[oR] = d2f(lam[oR]);
  }
}

// ---------------------------------------------------------------------------------
// growth matrix M = M1 - M2 and sigma_1 ("Energy analysis")
// ---------------------------------------------------------------------------------
template <class T>
struct Prim {
  T rho, u[3], p, a, b;
};

// fb = 1/sqrt(gamma), fa = sqrt((gamma-1)/gamma): b = fb c, a = fa c
template <class T>
__device__ __forceinline__ Prim<T> prim_at(const T* __restrict__ w, size_t o, long long cells,
                                           T gamma, T fb, T fa) {
  Prim<T> P;
  P.rho = w[o];
  const T ir = T(1) / P.rho;
  P.u[0] = w[o + cells] * ir;
  P.u[1] = w[o + 2 * cells] * ir;
  P.u[2] = w[o + 3 * cells] * ir;
  P.p = (gamma - T(1)) * (w[o + 4 * cells] - T(0.5) * P.rho * (P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]));
  const T cs = sqrt(gamma * P.p * ir);
  P.b = fb * cs;
  P.a = fa * cs;
  return P;
}

// Largest eigenvalue of a symmetric positive semidefinite N x N matrix: Householder
// reduction to tridiagonal form, then Laguerre's iteration on the characteristic
// polynomial of the tridiagonal matrix from a Gershgorin upper bound.  For a
// polynomial with only real roots Laguerre's iteration started to the right of the
// largest root decreases monotonically to it (cubically near a simple root), so a
// fixed small number of steps suffices.  The matrix is scaled to unit trace first.
// Only the lower triangle of A is read and written: step k reflects the column below
// the diagonal onto its first entry (the off-diagonal alpha_k) and updates the trailing
// block A[k+1.., k+1..] by the symmetric rank-2 form A - 2 (v q^T + q v^T).
template <class T, int N>
__device__ T max_eig_sym(T A[N][N]) {
  T tr = T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) tr += A[i][i];
  if (!(tr > T(0))) return T(0);
  const T inv = T(1) / tr;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) A[i][j] *= inv;
  T off[N];   // off[i]: the entry (i+1, i) of the tridiagonal matrix
#pragma unroll
  for (int k = 0; k < N - 2; ++k) {
    T nrm2 = T(0);
#pragma unroll
    for (int i = k + 1; i < N; ++i) nrm2 += A[i][k] * A[i][k];
    const T x0 = A[k + 1][k];
    const T rest = nrm2 - x0 * x0;
    off[k] = x0;
    if (!(rest > T(0))) continue;              // column already reduced
    const T nrm = sqrt(nrm2);
    const T alpha = x0 >= T(0) ? -nrm : nrm;
    off[k] = alpha;
    T v[N];
#pragma unroll
    for (int i = k + 1; i < N; ++i) v[i] = A[i][k];
    v[k + 1] = x0 - alpha;
    const T sc = T(1) / sqrt(v[k + 1] * v[k + 1] + rest);
#pragma unroll
    for (int i = k + 1; i < N; ++i) v[i] *= sc;
    // p = B v over the trailing block B (lower triangle: B[i][j] = A[max][min])
    T q[N];
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      T acc = T(0);
#pragma unroll
      for (int j = k + 1; j < N; ++j) acc += (j <= i ? A[i][j] : A[j][i]) * v[j];
      q[i] = acc;
    }
    T vp = T(0);
#pragma unroll
    for (int i = k + 1; i < N; ++i) vp += v[i] * q[i];
#pragma unroll
    for (int i = k + 1; i < N; ++i) q[i] -= vp * v[i];
#pragma unroll
    for (int i = k + 1; i < N; ++i)
#pragma unroll
      for (int j = k + 1; j <= i; ++j) A[i][j] -= T(2) * (v[i] * q[j] + q[i] * v[j]);
  }
  off[N - 2] = A[N - 1][N - 2];
  T d[N], e2[N];
  T ub = T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    d[i] = A[i][i];
    const T bl = i > 0 ? fabs(off[i - 1]) : T(0);
    const T br = i < N - 1 ? fabs(off[i]) : T(0);
    e2[i] = i < N - 1 ? off[i] * off[i] : T(0);
    const T g = d[i] + bl + br;
    ub = g > ub ? g : ub;
  }
  T x = ub * T(1.0000002) + T(1e-30);
  const T n = T(N);
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    // p, p', p'' of det(T - x I) by the three-term recurrence
    T p0 = T(1), p1 = d[0] - x;
    T q0 = T(0), q1 = T(-1);
    T r0 = T(0), r1 = T(0);
#pragma unroll
    for (int i = 1; i < N; ++i) {
      const T dx = d[i] - x;
      const T p2 = dx * p1 - e2[i - 1] * p0;
      const T q2 = -p1 + dx * q1 - e2[i - 1] * q0;
      const T r2 = T(-2) * q1 + dx * r1 - e2[i - 1] * r0;
      p0 = p1; p1 = p2;
      q0 = q1; q1 = q2;
      r0 = r1; r1 = r2;
    }
    if (p1 == T(0)) break;
    const T ip = T(1) / p1;
    const T G = q1 * ip;
    const T H = G * G - r1 * ip;
    T disc = (n - T(1)) * (n * H - G * G);
    disc = disc > T(0) ? sqrt(disc) : T(0);
    const T den = G >= T(0) ? G + disc : G - disc;
    if (den == T(0)) break;
    const T step = n / den;
    x -= step;
    if (fabs(step) <= (sizeof(T) == 8 ? T(1e-15) : T(2e-7)) * fabs(x)) break;
  }
  return x * tr;
}

// sigma_1 of M: the square root of the largest eigenvalue of M^T M, on the full 5 x 5
// matrix (N = 5) or on its (rho, u1, u2, p) block for a 2D box (N = 4)
template <class T, int N>
__device__ T sigma1_of(const T M[5][5]) {
  constexpr int id5[5] = {0, 1, 2, 3, 4};
  constexpr int id4[4] = {0, 1, 2, 4};
  T B[N][N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = i; j < N; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int kk = N == 5 ? id5[k] : id4[k];
        acc += M[kk][N == 5 ? id5[i] : id4[i]] * M[kk][N == 5 ? id5[j] : id4[j]];
      }
      B[j][i] = acc;   // lower triangle (j >= i)
    }
  }
  const T l = max_eig_sym<T, N>(B);
  return sqrt(l > T(0) ? l : T(0));
}

// Growth matrix M = M1 - M2 of one cell from central differences of rho, u, p, a, b at
// its six neighbours (closed forms of section "Energy analysis").
template <class CT>
__device__ __forceinline__ void growth_matrix(const GridDesc& g, const Coef<CT>& c, const CT* __restrict__ w,
                                              int b, int x, int y, int z, CT M[5][5]) {
  const CT gam = c.gamma, gm1 = c.gm1;
  const size_t box = (size_t)b * 5 * g.cells;
  auto at = [&](int xx, int yy, int zz) {
    return box + (size_t)wrap(zz, g.nz) * g.plane + (size_t)wrap(yy, g.ny) * g.nx + wrap(xx, g.nx);
  };
  const CT fb = CT(1) / sqrt(gam), fa = sqrt(gm1 / gam);
  const Prim<CT> P0 = prim_at<CT>(w, at(x, y, z), g.cells, gam, fb, fa);
  Prim<CT> Pm[3], Pp[3];
  Pm[0] = prim_at<CT>(w, at(x - 1, y, z), g.cells, gam, fb, fa);
  Pp[0] = prim_at<CT>(w, at(x + 1, y, z), g.cells, gam, fb, fa);
  Pm[1] = prim_at<CT>(w, at(x, y - 1, z), g.cells, gam, fb, fa);
  Pp[1] = prim_at<CT>(w, at(x, y + 1, z), g.cells, gam, fb, fa);
  Pm[2] = prim_at<CT>(w, at(x, y, z - 1), g.cells, gam, fb, fa);
  Pp[2] = prim_at<CT>(w, at(x, y, z + 1), g.cells, gam, fb, fa);
  CT drho[3], du[3][3], dp[3], da[3], db[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const CT h = c.hidx[j];
    drho[j] = (Pp[j].rho - Pm[j].rho) * h;
    dp[j] = (Pp[j].p - Pm[j].p) * h;
    da[j] = (Pp[j].a - Pm[j].a) * h;
    db[j] = (Pp[j].b - Pm[j].b) * h;
#pragma unroll
    for (int k = 0; k < 3; ++k) du[k][j] = (Pp[j].u[k] - Pm[j].u[k]) * h;
  }
  const CT div = du[0][0] + du[1][1] + du[2][2];
  // M1 (closed form)
#pragma unroll
  for (int i2 = 0; i2 < 5; ++i2)
#pragma unroll
    for (int j2 = 0; j2 < 5; ++j2) M[i2][j2] = i2 == j2 ? CT(0.5) * div : CT(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    M[0][1 + j] = M[1 + j][0] = CT(0.5) * db[j];
    M[1 + j][4] = M[4][1 + j] = CT(0.5) * da[j];
  }
  // minus M2 (closed form)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    M[0][1 + j] -= P0.b / P0.rho * drho[j];
#pragma unroll
    for (int k = 0; k < 3; ++k) M[1 + k][1 + j] -= du[k][j];
    M[4][1 + j] -= CT(2) / gm1 * da[j];
    M[1 + j][4] -= P0.a / (CT(2) * P0.p) * dp[j];
  }
  M[0][4] -= sqrt(gm1) / CT(2) * div;
  M[4][4] -= gm1 / CT(2) * div;
}

// (hi, lo) += (bhi, blo) for unevaluated float pairs hi + lo: Knuth's two-sum of the high
// parts, the low parts added to its error, then a renormalising fast two-sum.  The pair
// keeps the sum of float terms to about 2^-44 relative; the result does not depend on
// the order of the two operands.
__device__ __forceinline__ void df_add(float& hi, float& lo, float bhi, float blo) {
  const float s = hi + bhi;
  const float bb = s - hi;
  float e = (hi - (s - bb)) + (bhi - bb);
  e = e + (lo + blo);
  hi = s + e;
  lo = e - (hi - s);
}

// sigma_1 by plane marching.  A CTA owns a TX x SG_TY tile of columns and a range of
// planes (march_range, as the stencil kernels); the primitives (rho, u1, u2, u3, p, a, b)
// of three consecutive planes of the tile and its one-cell halo sit in a shared-memory
// ring, filled from register-staged loads one plane ahead, so each state is loaded and
// converted once per CTA instead of seven times per cell.  The growth matrix of a cell
// is then the closed form of growth_matrix() on those values (the same operations, so the
// same sigma_1 bits).  Statistics: every CTA writes its (max, sum) for its box and zeros
// for the other boxes; the last CTA (ticket[0]) reduces them per box in a fixed order.
namespace sgk {
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int SY = TY + 2;
constexpr int SP = SX * SY;
constexpr int NV = 7;   // rho, u1, u2, u3, p, a, b
static_assert(SP <= 2 * NT, "a plane must fit two load rounds");
}  // namespace sgk

size_t sigma1_march_ctas_bound(const GridDesc& g) {
  // the padded (bounded) box has one more column on each side
  const long long cols = (long long)((g.nx + 2 + TX - 1) / TX) * ((g.ny + 2 + sgk::TY - 1) / sgk::TY) * g.batch;
  return (size_t)(cols > 2048 ? cols : 2048);
}

template <class CT>
__global__ void __launch_bounds__(sgk::NT, sizeof(CT) == 4 ? 4 : 1) k_sigma1(GridDesc g, Coef<CT> c,
                                                                          const CT* __restrict__ w,
                                                                          float* __restrict__ sig, double* partial,
                                                                          double* stats, unsigned* ticket,
                                                                          NuRule rule, double* __restrict__ sigd) {
  using namespace sgk;
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* sP = reinterpret_cast<CT*>(smem_raw);   // [3][NV][SP]
  __shared__ double sh[32];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  int b, x0, y0, kz0, kz1;
  march_range<TX, TY>(g, b, x0, y0, kz0, kz1);
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < g.nx && gy < g.ny;
  const int cp = valid ? gy * g.nx + gx : 0;
  const size_t boxoff = (size_t)b * 5 * g.cells;
  const CT gam = c.gamma, gm1 = c.gm1;
  const CT fb = CT(1) / sqrt(gam), fa = sqrt(gm1 / gam);
  int ho[2];
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int t = tid + it * NT;
    const int ly = t / SX, lx = t - ly * SX;
    ho[it] = t < SP ? wrap(y0 + ly - 1, g.ny) * g.nx + wrap(x0 + lx - 1, g.nx) : 0;
  }
  auto load = [&](CT (&q)[2][5], int k) {
    const size_t pb = boxoff + (size_t)wrap(k, g.nz) * g.plane;
#pragma unroll
    for (int it = 0; it < 2; ++it)
      if (tid + it * NT < SP) {
#pragma unroll
        for (int v = 0; v < 5; ++v) q[it][v] = w[pb + v * (size_t)g.cells + ho[it]];
      }
  };
  auto store = [&](const CT (&q)[2][5], int slot) {
    CT* P = sP + slot * NV * SP;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int t = tid + it * NT;
      if (t < SP) {
        // the operations of prim_at()
        const CT rho = q[it][0];
        const CT ir = CT(1) / rho;
        const CT u0 = q[it][1] * ir, u1 = q[it][2] * ir, u2 = q[it][3] * ir;
        const CT p = (gam - CT(1)) * (q[it][4] - CT(0.5) * rho * (u0 * u0 + u1 * u1 + u2 * u2));
        const CT cs = sqrt(gam * p * ir);
        P[0 * SP + t] = rho;
        P[1 * SP + t] = u0;
        P[2 * SP + t] = u1;
        P[3 * SP + t] = u2;
        P[4 * SP + t] = p;
        P[5 * SP + t] = fa * cs;
        P[6 * SP + t] = fb * cs;
      }
    }
  };
  auto slot = [&](int k) { return (k - kz0 + 1) % 3; };
  {
    CT q0[2][5], q1[2][5], q2[2][5];
    load(q0, kz0 - 1);
    load(q1, kz0);
    load(q2, kz0 + 1);
    store(q0, slot(kz0 - 1));
    store(q1, slot(kz0));
    store(q2, slot(kz0 + 1));
  }
  __syncthreads();
  const int ic = (ty + 1) * SX + (tx + 1);
  CT vmax = CT(0);
  double vsum = 0.0;             // FP64 contexts
  float shi = 0.0f, slo = 0.0f;  // FP32 sigma_1: a compensated float-pair sum
  for (int k = kz0; k < kz1; ++k) {
    const bool more = k + 1 < kz1;
    CT qf[2][5];
    if (more) load(qf, k + 2);
    if (valid) {
      const CT* P0 = sP + slot(k) * NV * SP;
      const CT* Pm = sP + slot(k - 1) * NV * SP;
      const CT* Pp = sP + slot(k + 1) * NV * SP;
      // neighbour values of quantity v in direction j: (minus, plus)
      auto nb = [&](int v, int j, CT& m, CT& pl) {
        if (j == 0) {
          m = P0[v * SP + ic - 1];
          pl = P0[v * SP + ic + 1];
        } else if (j == 1) {
          m = P0[v * SP + ic - SX];
          pl = P0[v * SP + ic + SX];
        } else {
          m = Pm[v * SP + ic];
          pl = Pp[v * SP + ic];
        }
      };
      CT drho[3], du[3][3], dp[3], da[3], db[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const CT h = c.hidx[j];
        CT m, pl;
        nb(0, j, m, pl);
        drho[j] = (pl - m) * h;
        nb(4, j, m, pl);
        dp[j] = (pl - m) * h;
        nb(5, j, m, pl);
        da[j] = (pl - m) * h;
        nb(6, j, m, pl);
        db[j] = (pl - m) * h;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          nb(1 + kk, j, m, pl);
          du[kk][j] = (pl - m) * h;
        }
      }
      const CT rho0 = P0[0 * SP + ic], p0 = P0[4 * SP + ic], a0 = P0[5 * SP + ic], b0 = P0[6 * SP + ic];
      CT M[5][5];
      const CT div = du[0][0] + du[1][1] + du[2][2];
#pragma unroll
      for (int i2 = 0; i2 < 5; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 5; ++j2) M[i2][j2] = i2 == j2 ? CT(0.5) * div : CT(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        M[0][1 + j] = M[1 + j][0] = CT(0.5) * db[j];
        M[1 + j][4] = M[4][1 + j] = CT(0.5) * da[j];
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        M[0][1 + j] -= b0 / rho0 * drho[j];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) M[1 + kk][1 + j] -= du[kk][j];
        M[4][1 + j] -= CT(2) / gm1 * da[j];
        M[1 + j][4] -= a0 / (CT(2) * p0) * dp[j];
      }
      M[0][4] -= sqrt(gm1) / CT(2) * div;
      M[4][4] -= gm1 / CT(2) * div;
      const CT s1 = g.nz == 1 ? sigma1_of<CT, 4>(M) : sigma1_of<CT, 5>(M);
      const size_t o = (size_t)b * g.cells + (size_t)k * g.plane + cp;
      if (sigd) {
        // FP64 contexts: sigma_1 and the rule's viscosity kept in FP64
        const double sd = (double)s1;
        sigd[o] = sd;
        if (rule.nud)
          rule.nud[o] = nu_checked(sd > rule.taud ? rule.lamd * sd : 0.0, rule.limitd, rule.cap != 0, rule.err);
        vmax = fmax(vmax, s1);
        vsum += sd;
      } else {
        const float sf = (float)s1;
        sig[o] = sf;
        if (rule.nu)
          rule.nu[o] = nu_checked(sf > rule.tau ? rule.lam * sf : 0.0f, rule.limit, rule.cap != 0, rule.err);
        vmax = fmax(vmax, CT(sf));
        df_add(shi, slo, sf, 0.0f);
      }
    }
    __syncthreads();   // plane k-1 no longer read
    if (more) store(qf, slot(k - 1));
    __syncthreads();   // plane k+2 visible
  }
  if (!stats) return;
  const double bmax = block_reduce(vmax, sh, MaxOp());
  double bsum;
  if (sigd) {
    bsum = block_reduce(vsum, sh, AddOp());
  } else {
    // the warp's float pairs, one FP64 value per warp, added in order by thread 0
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      df_add(shi, slo, __shfl_xor_sync(0xffffffffu, shi, o), __shfl_xor_sync(0xffffffffu, slo, o));
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = widen(shi) + widen(slo);
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < NT / 32; ++i) t += sh[i];
      sh[0] = t;
    }
    __syncthreads();
    bsum = sh[0];
  }
  const int G = gridDim.x;
  if (tid < g.batch) {
    partial[(size_t)(2 * tid) * G + blockIdx.x] = tid == b ? bmax : 0.0;
    partial[(size_t)(2 * tid + 1) * G + blockIdx.x] = tid == b ? bsum : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(&ticket[0], 1u) == (unsigned)G - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last CTA: per box, a fixed-order reduction of every CTA's partials
  __threadfence();
  for (int bb = 0; bb < g.batch; ++bb) {
    double m = 0.0, t = 0.0;
    for (int j = tid; j < G; j += NT) {
      m = fmax(m, partial[(size_t)(2 * bb) * G + j]);
      t += partial[(size_t)(2 * bb + 1) * G + j];
    }
    m = block_reduce(m, sh, MaxOp());
    t = block_reduce(t, sh, AddOp());
    if (tid == 0) {
      stats[2 * bb] = m;
      stats[2 * bb + 1] = t / (double)g.cells;
    }
  }
  if (tid == 0) ticket[0] = 0u;
}

// v_hat = S^-T V^-T lam of one cell (closed form of w_hat = T^T v_hat, "Symmetrization")
template <class CT>
__device__ __forceinline__ void vhat_cell(const CT* __restrict__ w, const double* __restrict__ lam, size_t o,
                                          long long cells, CT gamma, CT v[5]) {
  const CT gm1 = gamma - CT(1);
  const CT r = w[o], ir = CT(1) / r;
  const CT u0 = w[o + cells] * ir, u1 = w[o + 2 * cells] * ir, u2 = w[o + 3 * cells] * ir;
  const CT uu = u0 * u0 + u1 * u1 + u2 * u2;
  const CT p = gm1 * (w[o + 4 * cells] - CT(0.5) * r * uu);
  const CT cs = sqrt(gamma * p * ir);
  const CT sg = sqrt(gamma);
  const CT l0 = cvt<CT>(lam[o]), l1 = cvt<CT>(lam[o + cells]), l2 = cvt<CT>(lam[o + 2 * cells]),
           l3 = cvt<CT>(lam[o + 3 * cells]), l4 = cvt<CT>(lam[o + 4 * cells]);
  const CT y0 = l0 + u0 * l1 + u1 * l2 + u2 * l3 + CT(0.5) * uu * l4;
  const CT y4 = l4 / gm1;
  v[0] = sg * r / cs * y0 + r * cs / sg * y4;
  v[1] = r * (l1 + u0 * l4);
  v[2] = r * (l2 + u1 * l4);
  v[3] = r * (l3 + u2 * l4);
  v[4] = r * cs * sqrt(gm1 / gamma) * y4;
}

// Label accumulation: acc += max(0, v_hat^T M v_hat) / |grad v_hat|^2 per cell; for a
// 2D box the (rho, u1, u2, p) block.
template <class CT>
__global__ void __launch_bounds__(RB) k_label(GridDesc g, Coef<CT> c, const CT* __restrict__ w,
                                              const double* __restrict__ lam, float* __restrict__ acc) {
  const long long i = (long long)blockIdx.x * RB + threadIdx.x;
  if (i >= g.cells * g.batch) return;
  const int b = (int)(i / g.cells);
  const long long r = i - (long long)b * g.cells;
  const int x = (int)(r % g.nx), y = (int)((r / g.nx) % g.ny), z = (int)(r / g.plane);
  const size_t box = (size_t)b * 5 * g.cells;
  auto at = [&](int xx, int yy, int zz) {
    return box + (size_t)wrap(zz, g.nz) * g.plane + (size_t)wrap(yy, g.ny) * g.nx + wrap(xx, g.nx);
  };
  CT M[5][5];
  growth_matrix<CT>(g, c, w, b, x, y, z, M);
  CT v[5];
  vhat_cell<CT>(w, lam, at(x, y, z), g.cells, c.gamma, v);
  const bool two_d = g.nz == 1;
  CT growth = CT(0);
#pragma unroll
  for (int p = 0; p < 5; ++p)
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (!(two_d && (p == 3 || q == 3))) growth += v[p] * M[p][q] * v[q];
  CT grad2 = CT(0);
  const int dd[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    CT vm[5], vp[5];
    vhat_cell<CT>(w, lam, at(x - dd[d][0], y - dd[d][1], z - dd[d][2]), g.cells, c.gamma, vm);
    vhat_cell<CT>(w, lam, at(x + dd[d][0], y + dd[d][1], z + dd[d][2]), g.cells, c.gamma, vp);
#pragma unroll
    for (int p = 0; p < 5; ++p) {
      if (two_d && p == 3) continue;
      const CT gd = (vp[p] - vm[p]) * c.hidx[d];
      grad2 += gd * gd;
    }
  }
  const CT rate = (growth > CT(0) ? growth : CT(0)) / (grad2 + CT(1e-30));
  acc[i] += (float)rate;
}


// ---------------------------------------------------------------------------------
// added adjoint viscosity: coefficient rule and the operator alone
// ---------------------------------------------------------------------------------
__global__ void k_nu_rule(long long n, const float* __restrict__ s1, float lam, float tau,
                          float limit_nu, float* __restrict__ nu, unsigned* err, bool cap) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = s1[i];
  nu[i] = nu_checked(s > tau ? lam * s : 0.0f, limit_nu, cap, err);
}

// the same rule in FP64 (FP64 contexts)
__global__ void k_nu_rule_f64(long long n, const double* __restrict__ s1, double lam, double tau,
                              double limit_nu, double* __restrict__ nu, unsigned* err, bool cap) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = s1[i];
  nu[i] = nu_checked(s > tau ? lam * s : 0.0, limit_nu, cap, err);
}

__global__ void k_visc_apply(GridDesc g, double ix2, double iy2, double iz2, double f_rho, double f_mom,
                             double f_en, const float* __restrict__ nu, const double* __restrict__ a,
                             double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = g.cells * g.batch;
  if (i >= tot) return;
  const long long b = i / g.cells, r = i - b * g.cells;
  const int x = (int)(r % g.nx), y = (int)((r / g.nx) % g.ny), z = (int)(r / g.plane);
  auto cell = [&](int xx, int yy, int zz) {
    return (size_t)wrap(zz, g.nz) * g.plane + (size_t)wrap(yy, g.ny) * g.nx + wrap(xx, g.nx);
  };
  const size_t c0 = cell(x, y, z);
  const size_t nb[6] = {cell(x - 1, y, z), cell(x + 1, y, z), cell(x, y - 1, z),
                        cell(x, y + 1, z), cell(x, y, z - 1), cell(x, y, z + 1)};
  const float* nub = nu + b * g.cells;
  const double nc = nub[c0];
  const double i2[3] = {ix2, iy2, iz2};
  for (int v = 0; v < 5; ++v) {
    const double* av = a + (size_t)b * 5 * g.cells + (size_t)v * g.cells;
    const double ac = av[c0];
    double L = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double nm = 0.5 * (nc + nub[nb[2 * d]]);
      const double np = 0.5 * (nc + nub[nb[2 * d + 1]]);
      L += (np * (av[nb[2 * d + 1]] - ac) - nm * (ac - av[nb[2 * d]])) * i2[d];
    }
    out[(size_t)b * 5 * g.cells + (size_t)v * g.cells + c0] += (v == 0 ? f_rho : (v == 4 ? f_en : f_mom)) * L;
  }
}

// ---------------------------------------------------------------------------------
// adjoint energy: v_hat = S^-T V^-T w_hat in closed form ("Symmetrization")
// ---------------------------------------------------------------------------------
template <class T, class TIN>
__device__ __forceinline__ T energy_cell(const TIN* __restrict__ w, const TIN* __restrict__ lam,
                                         size_t box, long long cells, long long i, T gamma) {
  const T gm1 = gamma - T(1), sg = sqrt(gamma), sgg = sqrt(gm1 / gamma);
  const T r = cvt<T>(w[box + i]), ir = T(1) / r;
  const T u0 = cvt<T>(w[box + cells + i]) * ir, u1 = cvt<T>(w[box + 2 * cells + i]) * ir,
          u2 = cvt<T>(w[box + 3 * cells + i]) * ir;
  const T uu = u0 * u0 + u1 * u1 + u2 * u2;
  const T p = gm1 * (cvt<T>(w[box + 4 * cells + i]) - T(0.5) * r * uu);
  const T cs = sqrt(gamma * p * ir);
  const T l0 = cvt<T>(lam[box + i]), l1 = cvt<T>(lam[box + cells + i]), l2 = cvt<T>(lam[box + 2 * cells + i]),
          l3 = cvt<T>(lam[box + 3 * cells + i]), l4 = cvt<T>(lam[box + 4 * cells + i]);
  // y = V^-T lam, V^-1 = dw/dq
  const T y0 = l0 + u0 * l1 + u1 * l2 + u2 * l3 + T(0.5) * uu * l4;
  const T y1 = r * (l1 + u0 * l4), y2 = r * (l2 + u1 * l4), y3 = r * (l3 + u2 * l4);
  const T y4 = l4 / gm1;
  // v_hat = S^-T y
  const T v0 = sg * r / cs * y0 + r * cs / sg * y4;
  const T v4 = r * cs * sgg * y4;
  return v0 * v0 + y1 * y1 + y2 * y2 + y3 * y3 + v4 * v4;
}


// E[b] = dV sum_cells |v_hat|^2; the last block of each box adds the block partials in
// fixed order (ticket: per-box counters, zero on entry and on exit).
template <class T, class TIN>
__global__ void __launch_bounds__(RB, sizeof(T) == 4 ? 8 : 1) k_energy(GridDesc g, double gamma, double dV, const TIN* __restrict__ w,
                                               const TIN* __restrict__ lam, double* partial, double* E,
                                               unsigned* err, unsigned* ticket) {
  pdl_enter();
  __shared__ double sh[32];
  __shared__ bool last;
  const int b = blockIdx.y;
  const size_t box = (size_t)b * 5 * g.cells;
  double acc = 0.0;
  if constexpr (sizeof(T) == 4) {
    // FP32 cell energies: compensated float-pair sums per thread and across the warp
    // (FP32 instructions; FP64 runs at a small fraction of their rate), one FP64 value
    // per warp, the warps' values added in order by thread 0
    float hi = 0.0f, lo = 0.0f;
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < g.cells; i += (long long)gridDim.x * RB)
      df_add(hi, lo, energy_cell<T, TIN>(w, lam, box, g.cells, i, T(gamma)), 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      df_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = widen(hi) + widen(lo);
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < RB / 32; ++i) acc += sh[i];
    __syncthreads();   // sh is reused by the last block's reduction
  } else {
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < g.cells; i += (long long)gridDim.x * RB)
      acc += energy_cell<T, TIN>(w, lam, box, g.cells, i, T(gamma));
    acc = block_reduce(acc, sh, AddOp());
  }
  double* pb = partial + (size_t)b * gridDim.x;
  if (threadIdx.x == 0) {
    pb[blockIdx.x] = acc;
    __threadfence();
    last = atomicAdd(&ticket[b], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int j = threadIdx.x; j < (int)gridDim.x; j += RB) t += pb[j];
  t = block_reduce(t, sh, AddOp());
  if (threadIdx.x == 0) {
    const double v = t * dV;
    E[b] = v;
    if (!isfinite(v)) atomicOr(err, ERRBIT_NONFINITE);
    ticket[b] = 0u;
  }
}

__global__ void __launch_bounds__(RB) k_sum_partials(int nblk, double scale, const double* partial,
                                                     double* out, unsigned* err) {
  __shared__ double sh[RB];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += RB) s += partial[(size_t)b * nblk + i];
  s = block_reduce(s, sh, AddOp());
  if (threadIdx.x == 0) {
    const double v = s * scale;
    out[b] = v;
    if (err && !isfinite(v)) atomicOr(err, ERRBIT_NONFINITE);
  }
}

// ---------------------------------------------------------------------------------
// inner products with source shapes, source assembly, wave speed
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(RB) k_dot(const double* __restrict__ a, const double* __restrict__ phi,
                                            size_t n, double* partial) {
  __shared__ double sh[RB];
  const int m = blockIdx.y;
  const double* pm = phi + (size_t)m * n;
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB) s += a[i] * pm[i];
  s = block_reduce(s, sh, AddOp());
  if (threadIdx.x == 0) partial[(size_t)m * gridDim.x + blockIdx.x] = s;
}

__global__ void k_combine(const double* __restrict__ theta, const double* __restrict__ phi, int nphi,
                          size_t n, double* __restrict__ s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int m = 0; m < nphi; ++m) acc += theta[m] * phi[(size_t)m * n + i];
  s[i] = acc;
}

__global__ void __launch_bounds__(RB) k_max_wave(GridDesc g, double gamma, const double* __restrict__ w,
                                                 double* partial) {
  __shared__ double sh[RB];
  double mx = 0.0;
  const long long tot = g.cells * g.batch;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < tot; i += (long long)gridDim.x * RB) {
    const long long b = i / g.cells, r = i - b * g.cells;
    const size_t o = (size_t)b * 5 * g.cells + r;
    const double rho = w[o], ir = 1.0 / rho;
    const double u0 = w[o + g.cells] * ir, u1 = w[o + 2 * g.cells] * ir, u2 = w[o + 3 * g.cells] * ir;
    const double uu = u0 * u0 + u1 * u1 + u2 * u2;
    const double p = (gamma - 1.0) * (w[o + 4 * g.cells] - 0.5 * rho * uu);
    const double s = sqrt(uu) + sqrt(gamma * p * ir);
    mx = fmax(mx, isfinite(s) ? s : INFINITY);
  }
  mx = block_reduce(mx, sh, MaxOp());
  if (threadIdx.x == 0) partial[blockIdx.x] = mx;
}

__global__ void __launch_bounds__(RB) k_max_partials(int nblk, const double* partial, double* out) {
  __shared__ double sh[RB];
  double m = 0.0;
  for (int i = threadIdx.x; i < nblk; i += RB) m = fmax(m, partial[i]);
  m = block_reduce(m, sh, MaxOp());
  if (threadIdx.x == 0) out[0] = m;
}

__global__ void k_scale_boxes(GridDesc g, const double* __restrict__ seed, double* __restrict__ field) {
  const long long tot = g.cells * 5 * g.batch;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < tot) field[i] *= seed[i / (g.cells * 5)];
}

__global__ void __launch_bounds__(RB) k_dot_boxes(GridDesc g, const double* __restrict__ field, int comp,
                                                  const double* __restrict__ phi, double* partial) {
  __shared__ double sh[RB];
  const int m = blockIdx.y;
  const double* pm = phi + (size_t)m * g.cells;
  const long long tot = g.cells * g.batch;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < tot; i += (long long)gridDim.x * RB) {
    const long long b = i / g.cells, r = i - b * g.cells;
    s += field[(size_t)b * 5 * g.cells + (size_t)comp * g.cells + r] * pm[r];
  }
  s = block_reduce(s, sh, AddOp());
  if (threadIdx.x == 0) partial[(size_t)m * gridDim.x + blockIdx.x] = s;
}

// relative change of a sensitivity field: sum (b - a)^2 and sum b^2 over n elements
__global__ void __launch_bounds__(RB) k_diff_norms(const double* __restrict__ a, const double* __restrict__ b,
                                                   size_t n, double* partial) {
  __shared__ double sh[RB];
  double d2 = 0.0, b2 = 0.0;
  for (size_t i = (size_t)blockIdx.x * RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB) {
    const double bv = b[i], dv = bv - a[i];
    d2 += dv * dv;
    b2 += bv * bv;
  }
  d2 = block_reduce(d2, sh, AddOp());
  b2 = block_reduce(b2, sh, AddOp());
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = d2;
    partial[gridDim.x + blockIdx.x] = b2;
  }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  const size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (i + 1 < n) {
    const double2 v = *reinterpret_cast<const double2*>(in + i);
    *reinterpret_cast<float2*>(out + i) = make_float2(d2f(v.x), d2f(v.y));
  } else if (i < n) {
    out[i] = d2f(in[i]);
  }
}

}  // namespace

size_t diag_scratch_doubles(const GridDesc& g, int nphi) {
  size_t a = (size_t)2 * RG * g.batch + (size_t)2 * g.batch;
  if ((size_t)RGS * g.batch > a) a = (size_t)RGS * g.batch;
  if ((size_t)5 * RG * g.batch > a) a = (size_t)5 * RG * g.batch;
  if ((size_t)2 * RGS * g.batch > a) a = (size_t)2 * RGS * g.batch;
  // two-launch objective: partials, (N/D, sc) per box and 5 doubles per plane face
  const size_t ob = (size_t)2 * RG * g.batch + 2 * (size_t)g.batch + (size_t)g.ny * g.nz * g.batch * 5;
  if (ob > a) a = ob;
  // sigma_1 statistics: (max, sum) per box for every CTA of the plane-marching launch
  const size_t sg = 2 * sigma1_march_ctas_bound(g) * (size_t)g.batch;
  if (sg > a) a = sg;
  size_t b = (size_t)RG * (nphi > 0 ? nphi : 1);
  return (a > b ? a : b) + 64;
}

cudaError_t launch_objective(const GridDesc& g, double gamma, int plane_i, double pt_in,
                             const double* w, double weight, double* J_acc, double* lam,
                             unsigned* err, double* scratch, cudaStream_t st) {
  const int nf = g.ny * g.nz;
  int nblk = (nf + OB - 1) / OB;
  if (nblk > RG) nblk = RG;
  double* nd = scratch + (size_t)2 * RG * g.batch;
  k_obj_partial<<<dim3(nblk, g.batch), OB, 0, st>>>(g, gamma, plane_i, pt_in, w, scratch);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_obj_final<<<g.batch, RB, 0, st>>>(nblk, pt_in, weight, scratch, nd, J_acc, err);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess || !lam) return e;
  k_obj_grad<<<dim3(nblk, g.batch), OB, 0, st>>>(g, gamma, plane_i, pt_in, weight, w, nd, lam);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_objective_fast(const GridDesc& g, double gamma, int plane_i, double pt_in, const double* w,
                                  double weight, double* J_acc, double* lam, unsigned* err, double* scratch,
                                  unsigned* ticket, cudaStream_t st, float* lam_mirror) {
  const int nf = g.ny * g.nz;
  int nblk = (nf + OMB - 1) / OMB;
  if (nblk > RG) nblk = RG;
  double* partial = scratch;
  double* ndsc = scratch + (size_t)2 * RG * g.batch;
  double* aface = ndsc + 2 * (size_t)g.batch;
  cudaError_t e = launch_pdl(k_obj_sum, dim3(nblk, g.batch), dim3(OMB), 0, st, g, gamma, plane_i, pt_in, w, weight,
                             J_acc, lam != nullptr, err, partial, aface, ndsc, ticket);
  count_launch();
  if (e != cudaSuccess || !lam) return e;
  const long long n = (long long)nf * g.batch;
  e = launch_pdl(k_obj_scatter, dim3((unsigned)((n + 127) / 128)), dim3(128), 0, st, g, plane_i,
                 (const double*)aface, (const double*)ndsc, lam, lam_mirror);
  count_launch();
  return e;
}

cudaError_t launch_objective_sum(const GridDesc& g, double gamma, int plane_i, double pt_in, const double* w,
                                 double weight, double* J_acc, unsigned* err, double* scratch, unsigned* ticket,
                                 cudaStream_t st, const double** aface_out, const double** ndsc_out) {
  const int nf = g.ny * g.nz;
  int nblk = (nf + OMB - 1) / OMB;
  if (nblk > RG) nblk = RG;
  double* partial = scratch;
  double* ndsc = scratch + (size_t)2 * RG * g.batch;
  double* aface = ndsc + 2 * (size_t)g.batch;
  cudaError_t e = launch_pdl(k_obj_sum, dim3(nblk, g.batch), dim3(OMB), 0, st, g, gamma, plane_i, pt_in, w, weight,
                             J_acc, true, err, partial, aface, ndsc, ticket);
  count_launch();
  *aface_out = aface;
  *ndsc_out = ndsc;
  return e;
}

template <class CT>
cudaError_t launch_sigma1(const GridDesc& g, const Coef<CT>& c, const CT* w, float* sigma1,
                          double* stats, double* scratch, unsigned* ticket, cudaStream_t st,
                          const NuRule* rule, double* sigma1d) {
  const NuRule r = rule ? *rule : NuRule{0.f, 0.f, 0.f, nullptr, nullptr, 0.0, 0.0, 0.0, nullptr, 0};
  const size_t smem = sizeof(CT) * 3 * sgk::NV * sgk::SP;
  static MarchShape<TX, sgk::TY> shape;
  int ctas = 0;
  cudaError_t e = shape.get(k_sigma1<CT>, smem, g, nullptr, ctas);
  if (e != cudaSuccess) return e;
  if ((size_t)ctas > sigma1_march_ctas_bound(g)) return cudaErrorInvalidConfiguration;
  if (g.batch > sgk::NT) return cudaErrorInvalidConfiguration;
  e = launch_pdl(k_sigma1<CT>, dim3(ctas), dim3(sgk::NT), smem, st, g, c, w, sigma1, scratch, stats, ticket, r,
                 sigma1d);
  count_launch();
  return e;
}
template cudaError_t launch_sigma1<double>(const GridDesc&, const Coef<double>&, const double*, float*,
                                           double*, double*, unsigned*, cudaStream_t, const NuRule*, double*);
template cudaError_t launch_sigma1<float>(const GridDesc&, const Coef<float>&, const float*, float*,
                                          double*, double*, unsigned*, cudaStream_t, const NuRule*, double*);

template <class CT>
cudaError_t launch_label(const GridDesc& g, const Coef<CT>& c, const CT* w, const double* lam, float* acc,
                         cudaStream_t st) {
  const long long n = g.cells * g.batch;
  k_label<CT><<<(unsigned)((n + RB - 1) / RB), RB, 0, st>>>(g, c, w, lam, acc);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_label<double>(const GridDesc&, const Coef<double>&, const double*, const double*,
                                          float*, cudaStream_t);
template cudaError_t launch_label<float>(const GridDesc&, const Coef<float>&, const float*, const double*,
                                         float*, cudaStream_t);

cudaError_t launch_nu_rule(const GridDesc& g, const float* sigma1, double lambda, double tau,
                           double limit_nu, float* nu, unsigned* err, cudaStream_t st, bool cap) {
  const long long n = g.cells * g.batch;
  k_nu_rule<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, sigma1, (float)lambda, (float)tau,
                                                           (float)limit_nu, nu, err, cap);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_nu_rule_f64(const GridDesc& g, const double* sigma1, double lambda, double tau,
                               double limit_nu, double* nu, unsigned* err, cudaStream_t st, bool cap) {
  const long long n = g.cells * g.batch;
  k_nu_rule_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, sigma1, lambda, tau, limit_nu, nu, err, cap);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_visc_apply(const GridDesc& g, const double* idx2, const double* split, const float* nu,
                              const double* a, double* out, cudaStream_t st) {
  const long long n = g.cells * g.batch;
  k_visc_apply<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, idx2[0], idx2[1], idx2[2], split[0], split[1],
                                                            split[2], nu, a, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_energy(const GridDesc& g, double gamma, double dV, const double* w, const double* lam,
                          double* E, double* scratch, unsigned* err, bool fp32_transform, unsigned* ticket,
                          cudaStream_t st) {
  dim3 grid(RGS, g.batch);
  cudaError_t e = fp32_transform
                      ? launch_pdl(k_energy<float, double>, grid, dim3(RB), 0, st, g, gamma, dV, w, lam, scratch, E,
                                   err, ticket)
                      : launch_pdl(k_energy<double, double>, grid, dim3(RB), 0, st, g, gamma, dV, w, lam, scratch,
                                   E, err, ticket);
  count_launch();
  return e;
}

cudaError_t launch_energy_mirrors(const GridDesc& g, double gamma, double dV, const float* wf, const float* lamf,
                                  double* E, double* scratch, unsigned* err, unsigned* ticket, cudaStream_t st) {
  dim3 grid(RGS, g.batch);
  cudaError_t e = launch_pdl(k_energy<float, float>, grid, dim3(RB), 0, st, g, gamma, dV, wf, lamf, scratch, E, err,
                             ticket);
  count_launch();
  return e;
}

cudaError_t launch_dot(const double* a, const double* phi, int nphi, size_t n, double* out,
                       double* scratch, cudaStream_t st) {
  dim3 grid(RG, nphi);
  k_dot<<<grid, RB, 0, st>>>(a, phi, n, scratch);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials<<<nphi, RB, 0, st>>>(RG, 1.0, scratch, out, nullptr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_combine(const double* theta, const double* phi, int nphi, size_t n, double* s,
                           cudaStream_t st) {
  k_combine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, phi, nphi, n, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_max_wave(const GridDesc& g, double gamma, const double* w, double* out,
                            double* scratch, cudaStream_t st) {
  k_max_wave<<<RG, RB, 0, st>>>(g, gamma, w, scratch);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_max_partials<<<1, RB, 0, st>>>(RG, scratch, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ns

namespace ns {
cudaError_t launch_scale_boxes(const GridDesc& g, const double* seed, double* field, cudaStream_t st) {
  const long long tot = g.cells * 5 * g.batch;
  k_scale_boxes<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(g, seed, field);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dot_boxes(const GridDesc& g, const double* field, int comp, const double* phi, int nphi,
                             double* out, double* scratch, cudaStream_t st) {
  k_dot_boxes<<<dim3(RG, nphi), RB, 0, st>>>(g, field, comp, phi, scratch);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials<<<nphi, RB, 0, st>>>(RG, 1.0, scratch, out, nullptr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_diff_norms(const double* a, const double* b, size_t n, double* out2, double* scratch,
                              cudaStream_t st) {
  k_diff_norms<<<RG, RB, 0, st>>>(a, b, n, scratch);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials<<<2, RB, 0, st>>>(RG, 1.0, scratch, out2, nullptr);
  count_launch();
  return cudaGetLastError();
}

size_t objective_scratch_doubles(const GridDesc& g) {
  return (size_t)2 * RG * g.batch + (size_t)2 * g.batch;
}

cudaError_t launch_to_float(const double* in, float* out, size_t n, cudaStream_t st) {
  const size_t threads = (n + 1) / 2;
  k_to_float<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(in, out, n);
  count_launch();
  return cudaGetLastError();
}
}  // namespace ns
